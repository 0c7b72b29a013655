"""Pins of the oracle's error-analysis outputs, the tolerances of the
per-step GPU comparisons (tests/parity.py): the interpolant's slopes are
the derivatives of its interpolated gradient fields, the gross fields sum
the absolute contributions, and each CV's first-order rounding bound holds
for evaluations of the CV in binary32 on random configurations."""
import math

import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import synth

U32 = 2.0 ** -24


def _walker2d():
    spec = synth.mb64_specs(nw=1, stride=1)[0]
    return spec, oracle.Walker(spec)


def test_slopes_are_the_derivatives_of_the_interpolated_gradient():
    spec, w = _walker2d()
    f = w.new_field()
    r = np.random.default_rng(1)
    for _ in range(12):
        oracle.deposit(w, f, [r.uniform(0.5, 1.5), r.uniform(-3, 3)], r.uniform(0.2, 1.0))
    for _ in range(20):
        s = np.array([r.uniform(0.5, 1.5), r.uniform(-3, 3)])
        H, _ = oracle.interp_aux(w, f, s)
        for j in range(2):
            e = 1e-7
            sp, sm = s.copy(), s.copy()
            sp[j] += e
            sm[j] -= e
            # inside one cell the interpolant is multilinear: the central
            # difference is exact up to rounding unless it straddles a node
            fd = (oracle.interp(w, f, sp)[1] - oracle.interp(w, f, sm)[1]) / (2 * e)
            np.testing.assert_allclose(H[:, j], fd, rtol=1e-5, atol=1e-5 * np.abs(H).max())


def test_gross_fields_bound_the_net_fields():
    """The gross fields sum the absolute values of the contributions: after
    one hill A is the interpolated |field| (one contribution per node); after
    many overlapping hills the gross derivative fields exceed the net ones
    where the hills' slopes cancel, and never fall below them."""
    spec, w = _walker2d()
    frames = synth.SweepFrames(1, seed=4, period=(80, 120)).frames(0, 60)
    res1 = oracle.run([w], frames[:1], [0], 0, 1, error_model=True)
    _, A_net = oracle.interp_aux(w, res1["fields"][0], res1["s"][0, 0, :2])
    np.testing.assert_allclose(res1["A"][0, 0, :3], A_net, rtol=1e-14)
    res = oracle.run([w], frames, [0], 0, 60, error_model=True)
    A_final_net = oracle.interp_aux(w, res["fields"][0], res["s"][-1, 0, :2])[1]
    assert np.all(res["A"][-1, 0, :3] >= A_final_net * (1 - 1e-12))
    # hills alternately at 0.4 and 0.6 of a 1D axis (identity CV), read at
    # 0.5: their slopes cancel in the net derivative field, not in the gross
    spec1 = {"natoms": 1, "cvs": [{"type": "pos_x", "a": [0]}], "grid": synth.grid([0.0], [1.0], [101], [False]),
             "hill": synth.hill(1.0, [0.05], 1, 10.0)}
    w1 = oracle.Walker(spec1)
    xs = np.array([0.4, 0.6] * 5 + [0.5])
    fr = np.zeros((len(xs), 1, 3))
    fr[:, 0, 0] = xs
    rc = oracle.run([w1], fr, [0], 1, len(xs), error_model=True)  # from step 1: the last step deposits too
    net = abs(oracle.interp(w1, rc["fields"][0], [0.5])[1][0])
    assert rc["A"][-1, 0, 1] > 100 * max(net, 1e-12)


def _f32_com(x, ia, ib):
    x = x.astype(np.float32)
    def part(idx):
        r0 = x[idx[0]]
        acc = np.zeros(3, np.float32)
        w = np.float32(1.0 / len(idx))
        for i in idx:
            acc = acc + w * (x[i] - r0)
        return r0, acc
    ra, a = part(ia)
    rb, b = part(ib)
    d = (rb - ra) + (b - a)
    return float(np.sqrt(np.sum(d * d, dtype=np.float32)))


def _f32_dihedral(x, ia):
    p = x[list(ia)].astype(np.float32)
    b1, b2, b3 = p[1] - p[0], p[2] - p[1], p[3] - p[2]
    m, n = np.cross(b1, b2), np.cross(b2, b3)
    lb2 = np.sqrt(np.dot(b2, b2))
    return float(np.arctan2(np.float32(lb2 * np.dot(b1, n)), np.float32(np.dot(m, n))))


def _f32_cn(x, ia, ib, r0, box=None):
    xa = x[list(ia)].astype(np.float32)[:, None, :]
    xb = x[list(ib)].astype(np.float32)[None, :, :]
    d = xa - xb
    if box is not None:
        L = np.float32(box)
        d = d - L * np.floor(d / L + np.float32(0.5))
    q = np.sum(d * d, axis=-1, dtype=np.float32) * np.float32(1.0 / (r0 * r0))
    sw = np.float32(1.0) / (np.float32(1.0) + q * q * q)
    s = np.float32(0.0)
    for row in sw:  # sequential rows of partial sums, as a thread sums
        s = np.float32(s + np.float32(row.sum(dtype=np.float32)))
    return float(s)


def test_cv_rounding_bounds_hold_for_binary32_evaluations():
    r = np.random.default_rng(7)
    spec = synth.mb64_specs(nw=1)[0]
    w = oracle.Walker(spec)
    ratios = {"com": 0.0, "dih": 0.0}
    for trial in range(100):
        x = synth.SweepFrames(1, seed=trial).frames(int(r.integers(0, 5000)), 1)[0].astype(np.float64)
        s64 = oracle.cv_eval(w, 0, x)[0]
        s32 = _f32_com(x, spec["cvs"][0]["a"], spec["cvs"][0]["b"])
        ratios["com"] = max(ratios["com"], abs(s32 - s64) / (U32 * oracle.cv_round_bound(w, 0, x)))
        p64 = oracle.cv_eval(w, 1, x)[0]
        p32 = _f32_dihedral(x, spec["cvs"][1]["a"])
        dp = (p32 - p64 + math.pi) % (2 * math.pi) - math.pi
        ratios["dih"] = max(ratios["dih"], abs(dp) / (U32 * oracle.cv_round_bound(w, 1, x)))
    cn_spec = synth.uneven1000_specs(seed=2, nw=4, sizes_2d=(48,), n1d=200, n3d=20)
    tm = synth.uneven1000_templates(2, nw=4)
    ratios["cn"] = 0.0
    for sp, t in zip(cn_spec, tm):
        wc = oracle.Walker(sp)
        k = len(sp["cvs"]) - 1
        c = sp["cvs"][k]
        for j in range(5):
            x = t + r.normal(scale=0.02, size=t.shape)
            s64 = oracle.cv_eval(wc, k, x)[0]
            s32 = _f32_cn(x, c["a"], c["b"], c["r0"])
            ratios["cn"] = max(ratios["cn"], abs(s32 - s64) / (U32 * oracle.cv_round_bound(wc, k, x)))
    print("largest error / bound", ratios)
    assert all(v <= 1.0 for v in ratios.values()), ratios
