"""Pins of the oracle's mABP method with compact hills (SI "Streamlined bias
potential updates", Eqs. (apfm), (btraj-grad), (compacthill), (Cupdate)) and
of the RMSD CV (SI "Definition of the RMSD"), against closed forms, the
paper's printed numbers and properties that do not restate the oracle's own
formulas."""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.optimize import brentq

import oracle
from paper_1609_09833_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _spec(lo, hi, n, periodic, a, p=20, b=0.9, c=0.001, kT=2.5, stride=1, w=1.0, cvs=None, natoms=1):
    d = len(n)
    if cvs is None:
        cvs = [{"type": "pos_x", "a": [0]} for _ in range(d)]
    return {"natoms": natoms, "cvs": cvs, "grid": synth.grid(lo, hi, n, periodic),
            "hill": synth.mabp_hill(a, p, b, c, kT, stride, w)}


def _nodes(spec, k):
    g = spec["grid"]
    n = g["n"][k]
    if g["periodic"][k]:
        return g["lo"][k] + np.arange(n) * (g["hi"][k] - g["lo"][k]) / n
    return np.linspace(g["lo"][k], g["hi"][k], n)


# ---------------------------------------------------------------- the compact hill


@pytest.mark.parametrize("p", [1, 3, 20])
def test_compact_hill_shape(p):
    a = 0.7
    assert oracle.compact(0.0, a, p) == (1.0, 0.0)  # S(0) = 1: the e^p prefactor
    for u in (a, -a, 1.0000001 * a, 5 * a):
        assert oracle.compact(u, a, p)[0] == 0.0  # compact support
    us = np.linspace(1e-4 * a, 0.9 * a, 400)  # (nearer the edge S underflows to 0 in FP64)
    S = np.array([oracle.compact(u, a, p)[0] for u in us])
    assert np.all((S > 0) & (S < 1)) and np.all(np.diff(S) < 0)
    assert all(oracle.compact(-u, a, p)[0] == oracle.compact(u, a, p)[0] for u in us[::37])
    # derivative against a central difference
    for u in (0.1 * a, 0.5 * a, 0.8 * a, -0.3 * a):
        e = 1e-6
        fd = (oracle.compact(u + e, a, p)[0] - oracle.compact(u - e, a, p)[0]) / (2 * e)
        assert oracle.compact(u, a, p)[1] == pytest.approx(fd, rel=1e-6, abs=1e-10)


@pytest.mark.parametrize("p", [1, 2, 20])
def test_half_width_matches_the_paper(p):
    """The paper's width at half height, w_a = 2 a sqrt(ln 2 / (p + ln 2))."""
    a = 18.0
    u_half = brentq(lambda u: oracle.compact(u, a, p)[0] - 0.5, 1e-9, a * (1 - 1e-12), xtol=1e-14)
    assert 2 * u_half == pytest.approx(2 * a * math.sqrt(math.log(2) / (p + math.log(2))), rel=1e-12)


def test_gaussian_alpha_of_equal_half_width_golden():
    """SI "Convergence with S_a^p": for a = 18, p = 1 the Gaussian
    exp(-x^2/alpha^2) of equal width at half height has alpha = 13.833."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "compact_hill_alpha.txt")) if l[0] != "#"]
    for a, p, alpha in rows:
        a, p, alpha = float(a), int(p), float(alpha)
        u_half = brentq(lambda u: oracle.compact(u, a, p)[0] - 0.5, 1e-9, a * (1 - 1e-12), xtol=1e-14)
        # the Gaussian falls to 1/2 at x = alpha sqrt(ln 2)
        assert round(u_half / math.sqrt(math.log(2)), 3) == alpha


# ---------------------------------------------------------------- histogram update, Eq. (Cupdate)


def test_deposit_at_nearest_node_with_compact_support_2d():
    spec = _spec([-1.0, -math.pi], [1.0, math.pi], [41, 36], [False, True], a=[0.26, 0.9], p=2)
    w = oracle.Walker(spec)
    x0, x1 = _nodes(spec, 0), _nodes(spec, 1)
    D0, D1 = x0[1] - x0[0], x1[1] - x1[0]
    # u = 17.3 on axis 0 (nearest node 17), u = 35.7 on axis 1 (nearest node 36 = node 0, across the seam)
    s = [x0[0] + 17.3 * D0, x1[0] + 35.7 * D1]
    f = w.new_field()
    ic = oracle.deposit(w, f, s, 1.0)
    assert list(ic) == [17, 0]
    h = f[:, 0].reshape(36, 41)
    nz = np.argwhere(h > 0)
    # support: |node - centre| < a along both axes (minimum image on the periodic one)
    d0 = np.abs(nz[:, 1] - 17) * D0
    d1 = np.minimum(np.abs(nz[:, 0] - 0), 36 - np.abs(nz[:, 0] - 0)) * D1
    assert np.all(d0 < 0.26) and np.all(d1 < 0.9)
    # and every node closer than a along both axes received the hill
    n0 = sum(1 for o in range(-40, 41) if abs(o) * D0 < 0.26)
    n1 = sum(1 for o in range(-17, 19) if abs(o) * D1 < 0.9)
    assert len(nz) == n0 * n1 == 11 * 11
    # the value is the product of the one-dimensional hills centred on the node
    for j1, j0 in nz[::7]:
        u0 = (17 - j0) * D0
        u1 = ((0 - j1 + 18) % 36 - 18) * D1
        assert h[j1, j0] == pytest.approx(oracle.compact(u0, 0.26, 2)[0] * oracle.compact(u1, 0.9, 2)[0], rel=1e-13)


def test_derivative_fields_are_d_dxi_of_the_deposited_hill():
    """h'_k at a node equals the derivative along xi_k of S(xi* - xi), taken
    by a central difference of the continuous product hill."""
    spec = _spec([0.0, 0.0], [2.0, 3.0], [81, 61], [False, False], a=[0.3, 0.45], p=3)
    w = oracle.Walker(spec)
    x0, x1 = _nodes(spec, 0), _nodes(spec, 1)
    f = w.new_field()
    oracle.deposit(w, f, [x0[40] + 0.004, x1[30] - 0.01], 1.0)
    c0, c1 = x0[40], x1[30]

    def hill(p0, p1):
        return oracle.compact(c0 - p0, 0.3, 3)[0] * oracle.compact(c1 - p1, 0.45, 3)[0]

    e = 1e-6
    for j0, j1 in ((38, 30), (42, 27), (35, 33), (44, 31)):
        node = j0 + 81 * j1
        fd0 = (hill(x0[j0] + e, x1[j1]) - hill(x0[j0] - e, x1[j1])) / (2 * e)
        fd1 = (hill(x0[j0], x1[j1] + e) - hill(x0[j0], x1[j1] - e)) / (2 * e)
        assert f[node, 1] == pytest.approx(fd0, rel=1e-6, abs=1e-9)
        assert f[node, 2] == pytest.approx(fd1, rel=1e-6, abs=1e-9)
    # total mass: the sum over nodes approximates the product of the 1D integrals
    I0 = quad(lambda u: oracle.compact(u, 0.3, 3)[0], -0.3, 0.3)[0]
    I1 = quad(lambda u: oracle.compact(u, 0.45, 3)[0], -0.45, 0.45)[0]
    D0, D1 = x0[1] - x0[0], x1[1] - x1[0]
    assert f[:, 0].sum() * D0 * D1 == pytest.approx(I0 * I1, rel=1e-5)  # node sum of a smooth compact hill


def test_deposit_scales_with_height_and_adds():
    spec = _spec([-1.0], [1.0], [101], [False], a=[0.2], p=5)
    w = oracle.Walker(spec)
    f1, f2 = w.new_field(), w.new_field()
    oracle.deposit(w, f1, [0.1], 1.0)
    oracle.deposit(w, f2, [0.1], 0.25)
    oracle.deposit(w, f2, [0.1], 0.75)
    np.testing.assert_allclose(f2, f1, rtol=1e-15, atol=1e-300)


# ---------------------------------------------------------------- the bias, Eqs. (apfm) and (btraj-grad)


def test_bias_gradient_is_the_derivative_of_the_bias():
    """With h' the derivative of a smooth histogram h, the gradient of
    Eq. (btraj-grad) equals the derivative of the bias of Eq. (apfm): a
    central difference of V between neighbouring nodes."""
    spec = _spec([0.0], [4.0], [4001], [False], a=[0.1], b=0.85, c=0.02, kT=2.5)
    w = oracle.Walker(spec)
    xi = _nodes(spec, 0)
    h = 300.0 * np.exp(-((xi - 1.7) ** 2)) + 40.0 * xi
    hp = 300.0 * np.exp(-((xi - 1.7) ** 2)) * (-2.0 * (xi - 1.7)) + 40.0
    f = np.ascontiguousarray(np.stack([h, hp], axis=1))
    D = xi[1] - xi[0]
    for j in (300, 1500, 2200, 3500):
        Vm = oracle.lookup_mabp(w, f, [xi[j - 1]])[0]
        Vp = oracle.lookup_mabp(w, f, [xi[j + 1]])[0]
        V, dV, fl = oracle.lookup_mabp(w, f, [xi[j] + 0.3 * D])  # nearest node j
        assert fl == 0
        assert dV[0] == pytest.approx((Vp - Vm) / (2 * D), rel=1e-4)  # O(D^2) difference
        # limits of Eq. (apfm): linear for c (1-b) h << 1, logarithmic far above
    f0 = np.zeros((4001, 2))
    assert oracle.lookup_mabp(w, f0, [1.0])[0] == 0.0
    f0[:, 0] = 1e-9
    assert oracle.lookup_mabp(w, f0, [1.0])[0] == pytest.approx(2.5 * 0.85 * 0.02 * 1e-9, rel=1e-6)
    f0[:, 0] = 1e12
    assert oracle.lookup_mabp(w, f0, [1.0])[0] == pytest.approx(
        2.5 * 0.85 / 0.15 * math.log(0.02 * 0.15 * 1e12), rel=1e-9)


def test_lookup_is_nearest_node_and_limits_out_of_range():
    spec = _spec([0.0, -math.pi], [1.0, math.pi], [11, 8], [False, True], a=[0.25, 1.0], c=1.0, b=0.5, kT=1.0)
    w = oracle.Walker(spec)
    f = np.zeros((88, 3))
    f[:, 0] = np.arange(88)
    f[:, 1] = 1.0
    f[:, 2] = 2.0
    V, dV, fl = oracle.lookup_mabp(w, f, [0.34, -math.pi + 2.6 * 2 * math.pi / 8])  # nodes (3, 3)
    assert V == pytest.approx(math.log(0.5 * (3 + 11 * 3) + 1)) and fl == 0
    V, dV, fl = oracle.lookup_mabp(w, f, [1.3, math.pi - 0.1])  # axis 0 beyond its range -> node 10, axis 1 wraps to 0
    assert V == pytest.approx(math.log(0.5 * 10 + 1)) and fl == oracle.FLAG_OOR
    assert dV[0] == 0.0 and dV[1] == pytest.approx(1.0 * 0.5 * 1.0 * 2.0 / (1 + 0.5 * 10))  # c b kT h' / (1 + c (1-b) h)


# ---------------------------------------------------------------- RMSD


def test_rmsd_closed_forms_and_gradient():
    r = np.random.default_rng(3)
    N = 7
    x0 = r.normal(size=(N, 3))
    spec = {"natoms": N + 2, "cvs": [{"type": "rmsd", "a": np.arange(1, N + 1), "ref": x0}],
            "grid": synth.grid([0.0], [12.0], [480], [False]), "hill": synth.mabp_hill([0.25], 20, 0.9, 0.001)}
    w = oracle.Walker(spec)
    x = np.zeros((N + 2, 3))
    x[1:N + 1] = x0
    s, J, fl = oracle.cv_eval(w, 0, x)
    assert s == pytest.approx(0.1, rel=1e-15) and fl == 0 and np.all(J == 0)  # the offset's lower bound
    t = np.array([0.3, -0.4, 1.2])
    x[1:N + 1] = x0 + t
    assert oracle.cv_eval(w, 0, x)[0] == pytest.approx(math.sqrt(t @ t + 0.01), rel=1e-14)  # no fit
    x[1:N + 1] = x0
    x[4] += [0.0, 0.6, 0.0]
    assert oracle.cv_eval(w, 0, x)[0] == pytest.approx(math.sqrt(0.36 / N + 0.01), rel=1e-14)
    x = r.normal(size=(N + 2, 3))
    s, J, _ = oracle.cv_eval(w, 0, x)
    e = 1e-6
    for i, k in ((1, 0), (4, 2), (7, 1), (0, 0), (8, 2)):
        xp, xm = x.copy(), x.copy()
        xp[i, k] += e
        xm[i, k] -= e
        fd = (oracle.cv_eval(w, 0, xp)[0] - oracle.cv_eval(w, 0, xm)[0]) / (2 * e)
        assert J[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-10)


# ---------------------------------------------------------------- whole method


@pytest.mark.slow
def test_mabp_converges_to_minus_b_times_the_free_energy():
    """Closed-loop mABP with compact hills on U(s) = 5 (s^2-1)^2, identity
    CV: once c (1-b) h >> 1, V_b = -b F + C (the stationary point of
    Eq. (apfm) under sampling density exp(-(F + V_b)/kT)); here F = U. RMS of
    V_b + b U - C over [-1.4, 1.4] below 0.5 kT."""
    kT, b = 2.5, 0.9
    spec = _spec([-2.0], [2.0], [401], [False], a=[0.3], p=20, b=b, c=0.05, kT=kT, stride=1)
    w = oracle.Walker(spec)
    f = w.new_field()
    T = 1_500_000
    noise = synth.rng(4321).normal(size=(T, 1, 3))
    _, s_hist = oracle.langevin_double_well(w, f, np.array([[-1.0, 0.0, 0.0]]), T, dt=0.002, mu=1.0, kw=5.0,
                                            noise=noise)
    xi = _nodes(spec, 0)
    sel = (xi > -1.4) & (xi < 1.4)
    V = np.array([oracle.lookup_mabp(w, f, [v])[0] for v in xi[sel]])
    U = 5.0 * (xi[sel] ** 2 - 1.0) ** 2
    resid = V + b * U
    rms = np.sqrt(np.mean((resid - resid.mean()) ** 2))
    assert rms < 0.5 * kT, rms
    assert np.sum(np.diff(np.sign(s_hist)) != 0) > 100
