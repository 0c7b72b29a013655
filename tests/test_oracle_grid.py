"""Pins of the oracle's grid steps: hill deposit (a3), height (a2),
interpolation (a4) and the chain rule (a5), against closed forms and
properties that do not restate the oracle's own formulas."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_1609_09833_gb300 import synth


def _spec(lo, hi, n, periodic, sigma, w=1.0, gamma=10.0, kT=2.5, stride=1, cutoff=4.0, natoms=1, cvs=None):
    d = len(n)
    if cvs is None:
        cvs = [{"type": "pos_x", "a": [0]} for _ in range(d)]
    return {
        "natoms": natoms,
        "cvs": cvs,
        "grid": synth.grid(lo, hi, n, periodic),
        "hill": synth.hill(w, sigma, stride, gamma, kT, cutoff),
    }


def _nodes(spec, k):
    g = spec["grid"]
    n = g["n"][k]
    if g["periodic"][k]:
        return g["lo"][k] + np.arange(n) * (g["hi"][k] - g["lo"][k]) / n
    return np.linspace(g["lo"][k], g["hi"][k], n)


# ---------------------------------------------------------------- deposit


def test_single_hill_mass_peak_and_width_1d():
    """A hill of height h integrates to h sqrt(2 pi) sigma (times the erf
    mass of the 4-sigma box), peaks at the nearest node and has full width
    at half maximum 2 sqrt(2 ln 2) sigma."""
    sigma, h = 0.05, 1.7
    spec = _spec([-2.0], [2.0], [4001], [False], [sigma])
    w = oracle.Walker(spec)
    f = w.new_field()
    s0 = 0.123456
    oracle.deposit(w, f, [s0], h)
    xi = _nodes(spec, 0)
    D = 4.0 / 4000
    mass = f[:, 0].sum() * D
    R = w.halfwidth(0)
    assert R == 200
    # trapezoid on a 1e-3 grid is exact to ~1e-12 for this Gaussian; box = +-R nodes around the centre
    assert mass == pytest.approx(h * math.sqrt(2 * math.pi) * sigma * erf(4 / math.sqrt(2)), rel=5e-4)
    assert xi[np.argmax(f[:, 0])] == pytest.approx(s0, abs=D / 2)
    above = xi[f[:, 0] >= h / 2]
    assert above[-1] - above[0] == pytest.approx(2 * math.sqrt(2 * math.log(2)) * sigma, abs=2 * D)


def test_derivative_field_matches_fd_of_value_field():
    """The derivative fields equal central differences of the value field
    (catches a wrong sign or a wrong 1/sigma^2 factor)."""
    spec = _spec([-1.0, -1.0], [1.0, 1.0], [801, 601], [False, False], [0.08, 0.05])
    w = oracle.Walker(spec)
    f = w.new_field()
    oracle.deposit(w, f, [0.0371, -0.1234], 2.0)
    n0, n1 = 801, 601
    V = f[:, 0].reshape(n1, n0)
    d0 = f[:, 1].reshape(n1, n0)
    d1 = f[:, 2].reshape(n1, n0)
    D0, D1 = 2.0 / 800, 2.0 / 600
    fd0 = (V[:, 2:] - V[:, :-2]) / (2 * D0)
    fd1 = (V[2:, :] - V[:-2, :]) / (2 * D1)
    # compare away from the box edges where the truncation makes the FD jump
    inner = np.abs(V[1:-1, 1:-1]) > 1e-2
    np.testing.assert_allclose(d0[:, 1:-1][1:-1][inner], fd0[1:-1][inner], rtol=3e-3, atol=2e-3)
    np.testing.assert_allclose(d1[1:-1, :][:, 1:-1][inner], fd1[:, 1:-1][inner], rtol=3e-3, atol=2e-3)


def test_hill_is_separable_product_in_3d():
    """In 3D the hill factorises: V(i,j,k) V(i0,j0,k0)^2 = V(i,j0,k0) V(i0,j,k0) V(i0,j0,k)."""
    spec = _spec([0, 0, 0], [1, 1, 1], [33, 29, 31], [False, False, False], [0.06, 0.08, 0.05])
    w = oracle.Walker(spec)
    f = w.new_field()
    ic = oracle.deposit(w, f, [0.51, 0.47, 0.52], 1.0)
    V = f[:, 0].reshape(31, 29, 33)
    i0, j0, k0 = ic
    lhs = V * V[k0, j0, i0] ** 2
    rhs = V[k0, j0, :][None, None, :] * V[k0, :, i0][None, :, None] * V[:, j0, i0][:, None, None]
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-300)
    assert V[k0, j0, i0] == V.max()


def test_box_cutoff_integer_geometry():
    """Nodes receive a hill exactly inside the integer box |j - i_c| <= R,
    i_c = floor(u + 1/2), clipped at the ends of a non-periodic axis."""
    spec = _spec([0.0], [1.0], [101], [False], [0.02])
    w = oracle.Walker(spec)
    R = w.halfwidth(0)
    assert R == 8
    for s0, ic_expect in [(0.5, 50), (0.504999, 50), (0.505001, 51), (0.0, 0), (0.99, 99), (1.02, 102)]:
        f = w.new_field()
        ic = oracle.deposit(w, f, [s0], 1.0)
        assert ic[0] == ic_expect
        nz = np.nonzero(f[:, 0])[0]
        lo, hi = max(ic_expect - R, 0), min(ic_expect + R, 100)
        if lo > hi:
            assert nz.size == 0
        else:
            assert nz.min() == lo and nz.max() == hi


def test_periodic_hill_wraps_and_mirrors():
    """On a periodic axis a hill near -pi wraps onto nodes near +pi, and hills
    at -pi+e and pi-e are mirror images (value even, derivative odd)."""
    n = 64
    spec = _spec([-math.pi], [math.pi], [n], [True], [0.3])
    w = oracle.Walker(spec)
    e = 0.0137
    f1, f2 = w.new_field(), w.new_field()
    oracle.deposit(w, f1, [-math.pi + e], 1.0)
    oracle.deposit(w, f2, [math.pi - e], 1.0)
    mirror = (n - np.arange(n)) % n
    np.testing.assert_allclose(f1[:, 0], f2[mirror, 0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f1[:, 1], -f2[mirror, 1], rtol=1e-12, atol=1e-15)
    assert f1[n - 1, 0] > 0.5 and f1[n // 2, 0] == 0.0
    # a hill at s and at s + 2 pi are the same
    f3 = w.new_field()
    oracle.deposit(w, f3, [-math.pi + e + 2 * math.pi], 1.0)
    np.testing.assert_allclose(f3, f1, rtol=1e-12, atol=1e-15)


def test_periodic_brute_force_images():
    """Tiny periodic grid: every node's value equals the nearest-image Gaussian
    found by brute force over images, inside the box."""
    n = 16
    L = 2.0
    spec = _spec([0.0, 0.0], [L, 1.0], [n, 5], [True, False], [0.15, 0.2], cutoff=2.0)
    w = oracle.Walker(spec)
    f = w.new_field()
    s = np.array([1.93, 0.4])
    ic = oracle.deposit(w, f, s, 1.0)
    R0, R1 = w.halfwidth(0), w.halfwidth(1)
    xi0, xi1 = _nodes(spec, 0), _nodes(spec, 1)
    for j1 in range(5):
        for j0 in range(n):
            dmin = min((xi0[j0] + k * L - s[0] for k in (-1, 0, 1)), key=abs)
            ring = min(abs(j0 - ic[0] + k * n) for k in (-1, 0, 1))
            inside = ring <= R0 and abs(j1 - ic[1]) <= R1
            expect = math.exp(-dmin ** 2 / (2 * 0.15 ** 2) - (xi1[j1] - s[1]) ** 2 / (2 * 0.2 ** 2)) if inside else 0.0
            assert f[j1 * n + j0, 0] == pytest.approx(expect, rel=1e-12, abs=1e-300)


def test_periodic_stencil_must_not_wrap_onto_itself():
    with pytest.raises(ValueError):
        oracle.Walker(_spec([0.0], [1.0], [8], [True], [0.2]))


# ---------------------------------------------------------------- height


def test_height_closed_form():
    spec = _spec([0.0], [1.0], [11], [False], [0.1], w=1.3, gamma=10.0, kT=2.5)
    w = oracle.Walker(spec)
    # bias of dT ln 2 halves the height: dT = (gamma - 1) kT = 22.5
    assert oracle.height(w, 22.5 * math.log(2)) == pytest.approx(0.65, rel=1e-15)
    assert oracle.height(w, 0.0) == 1.3
    # hand-filled grid: V = c everywhere -> interpolated value is c
    f = w.new_field()
    f[:, 0] = 22.5 * math.log(4)
    V, dV, _ = oracle.interp(w, f, [0.37])
    assert oracle.height(w, V) == pytest.approx(1.3 / 4, rel=1e-14)


# ---------------------------------------------------------------- interpolation


def _multilinear_field(spec, coef, rng):
    """Fill every field with a function that is affine in each coordinate
    separately (exactly representable by multilinear interpolation)."""
    d = len(spec["grid"]["n"])
    axes = [_nodes(spec, k) for k in range(d)]
    mesh = np.meshgrid(*axes, indexing="ij")  # axis 0 fastest in the flat node index
    fields = []
    for q in range(1 + d):
        c = rng.normal(size=8)
        v = c[0] + sum(c[1 + k] * mesh[k] for k in range(d))
        if d >= 2:
            v = v + c[4] * mesh[0] * mesh[1]
        if d >= 3:
            v = v + c[5] * mesh[0] * mesh[2] + c[6] * mesh[1] * mesh[2] + c[7] * mesh[0] * mesh[1] * mesh[2]
        fields.append((v, c))
    flat = np.stack([fv.transpose(*reversed(range(d))).reshape(-1) for fv, _ in fields], axis=1)
    return np.ascontiguousarray(flat), fields


@pytest.mark.parametrize("d", [1, 2, 3])
def test_interp_exact_on_multilinear_fields(d):
    rng = np.random.default_rng(100 + d)
    n = [17, 13, 9][:d]
    spec = _spec([-1.0, 0.5, 2.0][:d], [1.0, 1.7, 3.0][:d], n, [False] * d, [0.3] * d)
    w = oracle.Walker(spec)
    flat, fields = _multilinear_field(spec, None, rng)
    for _ in range(20):
        s = np.array([rng.uniform(lo, hi) for lo, hi in zip(spec["grid"]["lo"], spec["grid"]["hi"])])
        V, dV, fl = oracle.interp(w, flat, s)
        assert fl == 0

        def ev(c):
            v = c[0] + sum(c[1 + k] * s[k] for k in range(d))
            if d >= 2:
                v += c[4] * s[0] * s[1]
            if d >= 3:
                v += c[5] * s[0] * s[2] + c[6] * s[1] * s[2] + c[7] * s[0] * s[1] * s[2]
            return v

        assert V == pytest.approx(ev(fields[0][1]), rel=1e-12, abs=1e-12)
        for k in range(d):
            assert dV[k] == pytest.approx(ev(fields[1 + k][1]), rel=1e-12, abs=1e-12)


def test_interp_at_nodes_periodic_and_clamp():
    rng = np.random.default_rng(7)
    spec = _spec([0.0, -math.pi], [2.0, math.pi], [9, 12], [False, True], [0.3, 0.3])
    w = oracle.Walker(spec)
    f = rng.normal(size=(9 * 12, 3))
    xi0, xi1 = _nodes(spec, 0), _nodes(spec, 1)
    for i, j in [(0, 0), (8, 11), (3, 5), (8, 0)]:
        V, dV, _ = oracle.interp(w, f, [xi0[i], xi1[j]])
        assert V == pytest.approx(f[j * 9 + i, 0], rel=1e-13)
        np.testing.assert_allclose(dV, f[j * 9 + i, 1:], rtol=1e-13)
    # periodic: s and s + 2 pi agree; between the last node and the first it blends them
    a = oracle.interp(w, f, [0.77, 3.0])
    b = oracle.interp(w, f, [0.77, 3.0 - 2 * math.pi])
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    mid = xi1[11] + 0.5 * (2 * math.pi / 12)
    V, _, _ = oracle.interp(w, f, [xi0[2], mid])
    assert V == pytest.approx(0.5 * (f[11 * 9 + 2, 0] + f[0 * 9 + 2, 0]), rel=1e-12)
    # outside a non-periodic range: value clamped, gradient along that axis zero
    V, dV, fl = oracle.interp(w, f, [2.5, xi1[4]])
    assert fl & oracle.FLAG_OOR
    assert V == pytest.approx(f[4 * 9 + 8, 0], rel=1e-13)
    assert dV[0] == 0.0 and dV[1] == pytest.approx(f[4 * 9 + 8, 2], rel=1e-13)


# ---------------------------------------------------------------- chain rule through a full step


def test_force_is_minus_gradient_of_interpolated_bias():
    """With an affine bias V = a + b.xi stored in the grid (derivative fields =
    b), the force of a non-deposit step equals minus the finite-difference
    gradient of V(s(x)) with respect to every atom coordinate."""
    rng = np.random.default_rng(21)
    specs = synth.mb64_specs(nw=1, stride=1000)
    spec = specs[0]
    w = oracle.Walker(spec)
    f = w.new_field()
    b = np.array([3.1, -0.7])
    xi0, xi1 = _nodes(spec, 0), _nodes(spec, 1)
    m0, m1 = np.meshgrid(xi0, xi1, indexing="xy")
    f[:, 0] = (0.4 + b[0] * m0 + b[1] * m1).reshape(-1)
    f[:, 1] = b[0]
    f[:, 2] = b[1]
    fr = synth.SweepFrames(1, seed=2).frames(0, 1).astype(np.float64)
    res = oracle.run([w], fr, [0], step0=1, T=1, fields=[f])
    assert res["flags"][0, 0] == 0
    F = res["F"][0]
    x = fr[0]

    def bias(xx):
        s = [oracle.cv_eval(w, k, xx)[0] for k in range(2)]
        return oracle.interp(w, f, s)[0]

    h = 1e-6
    for a in [0, 7, 16, 31, 32, 33, 34, 35]:
        for q in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, q] += h
            xm[a, q] -= h
            fd = (bias(xp) - bias(xm)) / (2 * h)
            assert F[a, q] == pytest.approx(-fd, rel=1e-5, abs=1e-7)
    # Newton's third law for CVs without external atoms
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)


def test_step_order_height_before_and_force_after_deposit():
    """Step 0 deposits a hill of height w (empty grid) and the step's V_b is
    read after the deposit; two walkers sharing one grid both take their
    heights from the grid before either deposit (Jacobi order)."""
    spec = _spec([-1.0], [1.0], [201], [False], [0.1], w=0.8, gamma=5.0, kT=2.0, stride=3)
    w = oracle.Walker(spec)
    x = np.array([[[0.25, 0.0, 0.0], [0.25, 0.0, 0.0]]])  # both walkers at s = 0.25 (node 125)
    shared = w.new_field()
    res = oracle.run([w, w], x, [0, 1], step0=0, T=1, fields=[shared, shared])
    assert list(res["deposits"]["height"]) == [0.8, 0.8]
    assert res["V"][0, 0] == pytest.approx(1.6, rel=1e-14)
    # next deposit step (3): height from V = 1.6 at the same point; dT = 8
    res = oracle.run([w, w], np.repeat(x, 4, axis=0), [0, 1], step0=1, T=4, fields=[shared, shared])
    assert list(res["deposits"]["step"]) == [3, 3]
    hh = 0.8 * math.exp(-1.6 / 8.0)
    np.testing.assert_allclose(res["deposits"]["height"], [hh, hh], rtol=1e-14)
    assert res["V"][-1, 0] == pytest.approx(1.6 + 2 * hh, rel=1e-14)
    # separate grids see only their own hill
    res = oracle.run([w, w], x, [0, 1], step0=0, T=1)
    assert res["V"][0, 0] == pytest.approx(0.8, rel=1e-14)


# ---------------------------------------------------------------- whole method


@pytest.mark.slow
def test_well_tempered_limit_on_double_well():
    """Closed-loop well-tempered run on U(s) = 5 (s^2-1)^2 with the identity
    CV: the bias converges to -(1 - 1/gamma) U + C (well-tempered limit cited
    by the paper for mABP/WTmetaD). RMS of V_b + (1-1/gamma) U - C over
    [-1.4, 1.4] must fall below 0.5 kT."""
    kT, gamma = 2.5, 10.0
    spec = _spec([-2.0], [2.0], [512], [False], [0.05], w=1.0, gamma=gamma, kT=kT, stride=100)
    w = oracle.Walker(spec)
    f = w.new_field()
    T = 2_000_000
    noise = synth.rng(12345).normal(size=(T, 1, 3))
    _, s_hist = oracle.langevin_double_well(w, f, np.array([[-1.0, 0.0, 0.0]]), T, dt=0.002, mu=1.0, kw=5.0,
                                            noise=noise)
    xi = _nodes(spec, 0)
    sel = (xi > -1.4) & (xi < 1.4)
    U = 5.0 * (xi ** 2 - 1.0) ** 2
    resid = f[sel, 0] + (1 - 1 / gamma) * U[sel]
    rms = np.sqrt(np.mean((resid - resid.mean()) ** 2))
    assert rms < 0.5 * kT, rms
    # and it did cross the barrier many times
    assert np.sum(np.diff(np.sign(s_hist)) != 0) > 100


# ---------------------------------------------------------------- CV range limit


def test_range_limit_wall_force_is_minus_gradient_of_its_energy():
    """The wall kwall/2 (s - smax)^2 above smax: on an empty bias the force on
    the atoms equals minus the finite-difference gradient of the wall energy
    of s(x) (COM distance CV), is zero below smax and continuous at it."""
    spec = _spec([0.0], [3.0], [301], [False], [0.05], natoms=4,
                 cvs=[{"type": "com_dist", "a": [0, 1], "b": [2, 3]}])
    spec["hill"] = synth.with_wall(spec["hill"], [1.2], 40.0)
    spec["hill"]["stride"] = 10 ** 9  # no hill: the force is the wall's alone
    w = oracle.Walker(spec)
    r = np.random.default_rng(2)
    x = np.concatenate([r.normal(scale=0.1, size=(2, 3)), r.normal(scale=0.1, size=(2, 3)) + [1.5, 0.2, 0.0]])
    res = oracle.run([w], x[None], [0], step0=1, T=1)
    s = res["s"][0, 0, 0]
    assert s > 1.2
    assert res["dV"][0, 0, 0] == pytest.approx(40.0 * (s - 1.2), rel=1e-12)

    def U(xx):
        sv = oracle.cv_eval(w, 0, xx)[0]
        return 0.5 * 40.0 * max(sv - 1.2, 0.0) ** 2

    e = 1e-6
    for a, k in ((0, 0), (2, 1), (3, 2)):
        xp, xm = x.copy(), x.copy()
        xp[a, k] += e
        xm[a, k] -= e
        assert res["F"][0, a, k] == pytest.approx(-(U(xp) - U(xm)) / (2 * e), rel=1e-6)
    # below the limit: no force; the wall starts from zero at smax
    x2 = x.copy()
    x2[2:] -= [0.5, 0.0, 0.0]
    res2 = oracle.run([w], x2[None], [0], step0=1, T=1)
    assert res2["s"][0, 0, 0] < 1.2 and np.all(res2["F"] == 0.0)
    spec0 = dict(spec, hill=dict(spec["hill"], kwall=0.0))
    res0 = oracle.run([oracle.Walker(spec0)], x[None], [0], step0=1, T=1)
    assert np.all(res0["F"] == 0.0)


def test_range_limit_adds_to_the_bias_gradient():
    spec = _spec([-2.0], [2.0], [401], [False], [0.1], w=1.0, stride=1)
    spec["hill"] = synth.with_wall(spec["hill"], [0.3], 25.0)
    w = oracle.Walker(spec)
    x = np.array([[0.55, 0.0, 0.0]])
    ref = oracle.run([oracle.Walker(_spec([-2.0], [2.0], [401], [False], [0.1], w=1.0, stride=1))], x[None], [0], 0, 1)
    res = oracle.run([w], x[None], [0], 0, 1)
    assert res["dV"][0, 0, 0] == pytest.approx(ref["dV"][0, 0, 0] + 25.0 * (0.55 - 0.3), rel=1e-12)
    assert res["V"][0, 0] == ref["V"][0, 0]  # V reports the bias alone
