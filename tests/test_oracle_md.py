"""Pins of the oracle's closed-loop dynamics (the model MD engine around the
force call): the Philox-4x32-10 counter generator against its published
known-answer values, the normals it feeds (standard and independent), the
two CV potentials against closed forms and the Mueller-Brown stationary
points of the literature, the move against the gradient of U(s(x)) and
the Einstein relation, and the whole closed loop against the well-tempered
limit of the COM-distance double well."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1609_09833_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(v, 16) for v in line.split()])
    return rows


def test_philox_known_answers_golden():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_uniform24_is_open_and_exact():
    assert oracle.uniform24(0) == 2.0 ** -25
    assert oracle.uniform24(0xFFFFFFFF) == 1.0 - 2.0 ** -25
    # only the top 24 bits matter, and the map is monotone
    assert oracle.uniform24(0x12345600) == oracle.uniform24(0x123456FF)
    assert oracle.uniform24(0x12345700) > oracle.uniform24(0x123456FF)


def test_normals_are_standard_and_independent():
    n = np.array([oracle.md_normals(99, s, t, a) for s in range(2) for t in range(200) for a in range(50)])
    assert n.shape == (20000, 3)
    for q in range(3):
        assert abs(n[:, q].mean()) < 5 / math.sqrt(len(n))
        assert abs(n[:, q].var() - 1.0) < 5 * math.sqrt(2.0 / len(n))
        assert stats.kstest(n[:, q], "norm").pvalue > 1e-4
    c = np.corrcoef(n.T)
    assert np.all(np.abs(c - np.eye(3)) < 5 / math.sqrt(len(n)))
    # a different stream, step, atom or seed gives different numbers
    base = oracle.md_normals(1, 2, 3, 4)
    for args in ((1, 2, 3, 5), (1, 2, 4, 4), (1, 3, 3, 4), (2, 2, 3, 4), (1, 2, 3 + (1 << 32), 4)):
        assert not np.allclose(oracle.md_normals(*args), base)


# Stationary points of the Mueller-Brown surface as tabulated in the
# literature (Mueller and Brown, Theor. Chim. Acta 53 (1979); coordinates to
# three decimals): three minima and two saddle points.
MB_MINIMA = [((-0.558, 1.442), -146.700), ((0.623, 0.028), -108.167), ((-0.050, 0.467), -80.768)]
MB_SADDLES = [((-0.822, 0.624), -40.665), ((0.212, 0.293), -72.249)]


def _mb_identity(scale=1.0):
    md = synth.md_muller_brown(scale=scale)
    md["mb"] = dict(md["mb"], map=(1.0, 0.0, 1.0, 0.0))
    return md


def _hess(md, p, e=1e-4):
    H = np.zeros((2, 2))
    for j in range(2):
        dp = np.zeros(2)
        dp[j] = e
        H[:, j] = (oracle.md_potential(md, p + dp)[1][:2] - oracle.md_potential(md, p - dp)[1][:2]) / (2 * e)
    return H


def test_muller_brown_stationary_points():
    md = _mb_identity()
    for (x, y), E in MB_MINIMA + MB_SADDLES:
        U, dU = oracle.md_potential(md, [x, y])
        assert U == pytest.approx(E, abs=0.02)
        # a stationary point to the precision of the tabulated coordinates
        H = _hess(md, np.array([x, y]))
        assert np.linalg.norm(dU[:2]) < 0.6e-3 * np.abs(np.linalg.eigvalsh(H)).max() * 2
    for (x, y), _ in MB_MINIMA:
        assert np.all(np.linalg.eigvalsh(_hess(md, np.array([x, y]))) > 0)
    for (x, y), _ in MB_SADDLES:
        ev = np.linalg.eigvalsh(_hess(md, np.array([x, y])))
        assert ev[0] < 0 < ev[1]


def test_potential_gradients_match_finite_differences():
    r = np.random.default_rng(3)
    for md in (synth.md_muller_brown(), synth.md_double_well(A=5.0, B=1.0)):
        for _ in range(20):
            s = np.array([r.uniform(0.3, 1.9), r.uniform(-3.0, 3.0)])
            U, dU = oracle.md_potential(md, s)
            for k in range(2):
                e = 1e-6
                sp, sm = s.copy(), s.copy()
                sp[k] += e
                sm[k] -= e
                fd = (oracle.md_potential(md, sp)[0] - oracle.md_potential(md, sm)[0]) / (2 * e)
                assert dU[k] == pytest.approx(fd, rel=1e-6, abs=1e-6 * (1 + abs(U)))
    dw = synth.md_double_well(A=5.0, B=1.0)
    assert oracle.md_potential(dw, [1.0])[0] == 0.0 and oracle.md_potential(dw, [-1.0])[0] == 0.0
    assert oracle.md_potential(dw, [0.0])[0] == pytest.approx(5.0)
    assert oracle.md_potential(synth.md_params(), [0.7, 0.1])[0] == 0.0


def _mb_walker():
    return synth.mb64_specs(nw=1, stride=10 ** 9)[0]  # no hill: the move sees only U


def test_move_follows_the_gradient_of_the_cv_potential():
    """With kT = 0 and no hill, one move is x - dt mu grad_x U(s(x)): checked
    against central differences of U(s(x)) in the atoms' coordinates."""
    spec = _mb_walker()
    w = oracle.Walker(spec)
    x = synth.SweepFrames(1, seed=3).frames(0, 1)[0].astype(np.float64)
    md = synth.md_muller_brown(mu=0.01, kT=0.0)
    res = oracle.run([w], x[None], [0], 1, 1, md=md, streams=[0])  # step 1: no hill
    step = res["Xn"][0] - x

    def U(xx):
        s = [oracle.cv_eval(w, k, xx)[0] for k in range(2)]
        return oracle.md_potential(md, s)[0]

    e = 1e-6
    for a in (0, 7, 20, 33, 35):
        for q in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a, q] += e
            xm[a, q] -= e
            g = (U(xp) - U(xm)) / (2 * e)
            assert step[a, q] == pytest.approx(-md["dt"] * md["mu"] * g, rel=1e-5, abs=1e-12)


def test_free_diffusion_obeys_the_einstein_relation():
    """No bias, no potential: every atom diffuses with D = mu kT, so the mean
    squared displacement after T steps is 6 mu kT T dt."""
    spec = dict(_mb_walker())
    w = oracle.Walker(spec)
    x0 = synth.SweepFrames(1, seed=4).frames(0, 1)[0].astype(np.float64)
    md = synth.md_params(dt=0.002, mu=0.3, kT=2.5, seed=11)
    T = 400
    disp = []
    for stream in range(20):
        res = oracle.md_run([w], x0, [0], md, [stream], 1, T)  # from step 1: no hill (stride 1e9)
        disp.append(res["x"] - x0)
    msd = np.mean(np.sum(np.concatenate(disp) ** 2, axis=1))
    expect = 6 * md["mu"] * md["kT"] * T * md["dt"]
    assert msd == pytest.approx(expect, rel=0.05)


@pytest.mark.slow
def test_closed_loop_com_distance_well_tempered_limit():
    """The one-walker FP64 workload closed: two 8-atom groups, COM distance s
    on U(s) = 5 (s^2 - 1)^2, overdamped Langevin of every atom (mu = 1, kT =
    2.5, dt = 0.002), well-tempered hills (gamma = 10). The distance of two
    freely diffusing centres in 3D has the free energy F(s) = U(s) - 2 kT ln s
    (the radial Jacobian), and the bias converges to -(1 - 1/gamma) F + C:
    RMS of V_b + (1 - 1/gamma) F - C over [0.3, 1.7] below 0.5 kT after 2e5
    steps."""
    kT, gamma = 2.5, 10.0
    spec = synth.double_well_com_spec()
    w = oracle.Walker(spec)
    md = synth.md_double_well(seed=7)
    res = oracle.md_run([w], synth.double_well_com_coords(21), [0], md, [3], 0, 200_000)
    xi = np.linspace(-2.0, 2.0, 512)
    sel = (xi > 0.3) & (xi < 1.7)
    F = 5.0 * (xi[sel] ** 2 - 1.0) ** 2 - 2.0 * kT * np.log(xi[sel])
    resid = res["fields"][0][sel, 0] + (1 - 1 / gamma) * F
    rms = np.sqrt(np.mean((resid - resid.mean()) ** 2))
    assert rms < 0.5 * kT, rms
    s = res["s"][:, 0, 0]
    assert s.min() < 0.4 and s.max() > 1.6  # the sampled range covers the window
