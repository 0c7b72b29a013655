"""Pins of the oracle's collective variables (step a1) against closed forms,
finite differences, invariances and exact rational arithmetic."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _walker(cvs, natoms, d=None):
    d = len(cvs)
    return oracle.Walker({
        "natoms": natoms,
        "cvs": cvs,
        "grid": {"lo": [-10.0] * d, "hi": [10.0] * d, "n": [64] * d, "periodic": [False] * d},
        "hill": {"w": 1.0, "sigma": [1.0] * d, "cutoff": 4.0, "gamma": 10.0, "kT": 2.5, "stride": 1},
    })


def _fd_jacobian(w, k, x, h=1e-6):
    J = np.zeros_like(x)
    for a in range(x.shape[0]):
        for q in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[a, q] += h
            xm[a, q] -= h
            J[a, q] = (oracle.cv_eval(w, k, xp)[0] - oracle.cv_eval(w, k, xm)[0]) / (2 * h)
    return J


def _rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


# ---------------------------------------------------------------- COM distance


def test_com_distance_closed_form():
    # group A: vertices of a cube centred at cA; group B: octahedron centred at cB
    cA = np.array([0.3, -0.2, 0.5])
    cB = np.array([1.3, 0.8, -0.5])
    cube = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], dtype=float) * 0.1
    octa = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=float) * 0.2
    x = np.concatenate([cA + cube, cB + octa])
    w = _walker([{"type": "com_dist", "a": np.arange(8), "b": np.arange(8, 14)}], 14)
    s, J, fl = oracle.cv_eval(w, 0, x)
    assert fl == 0
    assert s == pytest.approx(math.sqrt(3.0), rel=1e-15)
    # each A atom pulls with -1/8 u, each B atom with +1/6 u, u the unit separation
    u = (cB - cA) / math.sqrt(3.0)
    np.testing.assert_allclose(J[:8], np.tile(-u / 8, (8, 1)), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(J[8:], np.tile(u / 6, (6, 1)), rtol=1e-14, atol=1e-15)


def test_com_distance_masses_closed_form():
    # two atoms per group, masses 1 and 3: COM at 3/4 of the way
    x = np.array([[0, 0, 0], [4, 0, 0], [0, 2, 0], [0, 6, 0]], dtype=float)
    w = _walker([{"type": "com_dist", "a": [0, 1], "b": [2, 3], "ma": [1.0, 3.0], "mb": [3.0, 1.0]}], 4)
    s, J, _ = oracle.cv_eval(w, 0, x)
    # R_A = (3, 0, 0), R_B = (0, 3, 0)
    assert s == pytest.approx(3 * math.sqrt(2), rel=1e-15)
    u = np.array([-3.0, 3.0, 0.0]) / (3 * math.sqrt(2))
    np.testing.assert_allclose(J[0], -0.25 * u, rtol=1e-14)
    np.testing.assert_allclose(J[1], -0.75 * u, rtol=1e-14)
    np.testing.assert_allclose(J[2], 0.75 * u, rtol=1e-14)
    np.testing.assert_allclose(J[3], 0.25 * u, rtol=1e-14)


def test_com_distance_fd_and_invariance():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 3, size=(16, 3))
    w = _walker([{"type": "com_dist", "a": np.arange(8), "b": np.arange(8, 16),
                  "ma": rng.uniform(1, 16, 8), "mb": rng.uniform(1, 16, 8)}], 16)
    s, J, _ = oracle.cv_eval(w, 0, x)
    np.testing.assert_allclose(J, _fd_jacobian(w, 0, x), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(J.sum(axis=0), 0.0, atol=1e-14)
    R = _rot(rng)
    s2, _, _ = oracle.cv_eval(w, 0, x @ R.T + np.array([5.0, -2.0, 1.0]))
    assert s2 == pytest.approx(s, rel=1e-13)


def test_com_distance_min_image():
    box = (3.0, 4.0, 5.0)
    x = np.array([[0.1, 0.2, 0.3], [2.9, 3.9, 4.8]])  # separation (-0.2, -0.3, -0.5) through the faces
    w = _walker([{"type": "com_dist", "a": [0], "b": [1], "pbc": True, "box": box}], 2)
    s, _, _ = oracle.cv_eval(w, 0, x)
    assert s == pytest.approx(math.sqrt(0.2 ** 2 + 0.3 ** 2 + 0.5 ** 2), rel=1e-12)


# ---------------------------------------------------------------- dihedral


def _dihedral_geometry(phi, rng=None):
    """x2 at the origin, x3 on +z, x1 along +x, x4 rotated by +phi about +z:
    the IUPAC dihedral is phi by construction."""
    x = np.array([[1.0, 0, 0], [0, 0, 0], [0, 0, 1.2], [0.7 * math.cos(phi), 0.7 * math.sin(phi), 1.2]])
    # shift x1, x4 along the axis so bond angles are not 90 degrees (the dihedral does not change)
    x[0, 2] -= 0.4
    x[3, 2] += 0.3
    if rng is not None:
        x = x @ _rot(rng).T + rng.normal(size=3)
    return x


@pytest.mark.parametrize("phi", [0.0, math.pi / 2, -math.pi / 2, 2.5, -3.0, 1e-3, math.pi - 1e-9])
def test_dihedral_closed_form(phi):
    w = _walker([{"type": "dihedral", "a": [0, 1, 2, 3]}], 4)
    s, _, _ = oracle.cv_eval(w, 0, _dihedral_geometry(phi))
    assert s == pytest.approx(phi, abs=1e-13)
    s2, _, _ = oracle.cv_eval(w, 0, _dihedral_geometry(phi, np.random.default_rng(5)))
    assert s2 == pytest.approx(phi, abs=1e-12)


def test_dihedral_trans_is_pi_and_mirror_flips_sign():
    w = _walker([{"type": "dihedral", "a": [0, 1, 2, 3]}], 4)
    s, _, _ = oracle.cv_eval(w, 0, _dihedral_geometry(math.pi))
    assert abs(s) == pytest.approx(math.pi, abs=1e-13)
    x = _dihedral_geometry(1.1, np.random.default_rng(9))
    s1, _, _ = oracle.cv_eval(w, 0, x)
    s2, _, _ = oracle.cv_eval(w, 0, x * np.array([-1.0, 1.0, 1.0]))
    assert s2 == pytest.approx(-s1, abs=1e-13)


def test_dihedral_fd_sum_and_torque():
    rng = np.random.default_rng(11)
    w = _walker([{"type": "dihedral", "a": [3, 0, 2, 1]}], 5)
    for _ in range(5):
        x = rng.uniform(0, 1, size=(5, 3))
        s, J, fl = oracle.cv_eval(w, 0, x)
        assert fl == 0
        np.testing.assert_allclose(J, _fd_jacobian(w, 0, x), rtol=2e-6, atol=1e-8)
        np.testing.assert_allclose(J.sum(axis=0), 0.0, atol=1e-12)
        np.testing.assert_allclose(np.cross(x, J).sum(axis=0), 0.0, atol=1e-11)
        assert np.all(J[4] == 0.0)


# ---------------------------------------------------------------- coordination number


def _switch_exact(r: Fraction, n: int, m: int) -> Fraction:
    x = r
    return (1 - x ** n) / (1 - x ** m)


@pytest.mark.parametrize("n,m", [(6, 12), (6, 10), (8, 12)])
def test_switch_rational_arithmetic(n, m):
    for num, den in [(1, 3), (1, 2), (3, 4), (9, 10), (11, 10), (3, 2), (2, 1), (7, 2)]:
        x = Fraction(num, den)
        v, _ = oracle.switch(float(x), n, m)
        assert v == pytest.approx(float(_switch_exact(x, n, m)), rel=1e-13)
    # derivative against central differences away from x = 1
    for x in [0.3, 0.8, 1.3, 2.2]:
        _, d = oracle.switch(x, n, m)
        h = 1e-6
        fd = (oracle.switch(x + h, n, m)[0] - oracle.switch(x - h, n, m)[0]) / (2 * h)
        assert d == pytest.approx(fd, rel=1e-7)


def test_switch_special_points():
    assert oracle.switch(1.0, 6, 12)[0] == 0.5           # removable point r = r0
    assert oracle.switch(2.0, 6, 12)[0] == pytest.approx(1.0 / 65.0, rel=1e-15)
    assert oracle.switch(0.0, 6, 12)[0] == 1.0
    # limit n/m and slope n(n-m)/(2m) at x = 1 for the general formula
    v, d = oracle.switch(1.0, 6, 10)
    assert v == pytest.approx(0.6) and d == pytest.approx(-1.2)
    assert oracle.switch(1.0, 6, 12)[1] == pytest.approx(-1.5)


def test_coordination_closed_form_pairs():
    r0 = 0.4
    # ligand atom at origin, pocket atoms at r0 and 2 r0 along different axes
    x = np.array([[0, 0, 0], [r0, 0, 0], [0, 2 * r0, 0], [0, 0, 1e3]], dtype=float)
    w = _walker([{"type": "coord", "a": [0], "b": [1, 2, 3], "r0": r0, "n": 6, "m": 12}], 4)
    s, J, _ = oracle.cv_eval(w, 0, x)
    assert s == pytest.approx(0.5 + 1.0 / 65.0 + 1.0 / (1.0 + (1e3 / r0) ** 6), rel=1e-14)
    # d sw/dr at r0 is -1.5/r0 along +x for the pocket atom
    assert J[1, 0] == pytest.approx(-1.5 / r0, rel=1e-13)


def test_coordination_fd_sum_and_pbc():
    rng = np.random.default_rng(17)
    box = (2.0, 2.0, 2.0)
    x = rng.uniform(0, 2.0, size=(12, 3))
    cv = {"type": "coord", "a": np.arange(4), "b": np.arange(4, 12), "r0": 0.4, "n": 6, "m": 12, "pbc": True, "box": box}
    w = _walker([cv], 12)
    s, J, _ = oracle.cv_eval(w, 0, x)
    np.testing.assert_allclose(J, _fd_jacobian(w, 0, x), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(J.sum(axis=0), 0.0, atol=1e-13)
    # shifting any atom by a box vector leaves the minimum-image CN unchanged
    x2 = x.copy()
    x2[5] += np.array([2.0, -2.0, 4.0])
    x2[1] -= np.array([0.0, 2.0, 0.0])
    assert oracle.cv_eval(w, 0, x2)[0] == pytest.approx(s, rel=1e-13)
    # brute force over the 27 neighbouring images picks the same nearest pairs
    tot = 0.0
    for i in range(4):
        for j in range(4, 12):
            best = min(np.linalg.norm(x[i] - x[j] + np.array([a, b, c]) * 2.0)
                       for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
            tot += 1.0 / (1.0 + (best / 0.4) ** 6)
    assert s == pytest.approx(tot, rel=1e-12)
