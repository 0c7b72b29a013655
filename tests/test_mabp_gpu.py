"""GPU parity of the mABP method with compact S_a^p hills (SI "Streamlined
bias potential updates": Eqs. (apfm), (btraj-grad), (compacthill),
(Cupdate)) and of the RMSD CV (SI "Definition of the RMSD") against the FP64
oracle, in the windowed and per-step fused forms and the plain form.

mABP reads the bias at the nearest node, so a step whose CV lies within the
tie band of a half-node may read a neighbouring node on one side: such steps
are left out of the force comparison (and counted), as deposits whose
centre ties are (tests/parity.py). The band of a step is 4 |u32 - u64| +
1e-6 with |u32 - u64| bounded by the CV's rounding bound (the oracle's
error model) over the node spacing."""
import math

import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import synth
from tests import parity as P
from tests.test_parity_gpu import gpu_replay, oracle_replay

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import abp as A
    from paper_1609_09833_gb300 import build

    build.build()
    A.load()
    return A


@pytest.fixture()
def ctx(abp):
    c = abp.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _mabp(specs, a_bins=10.0, p=20, b=0.9, c=0.05, stride=1, w=1.0):
    out = []
    for sp in specs:
        sp = dict(sp)
        g = sp["grid"]
        a = [synth.bins(g, k, a_bins) for k in range(len(g["n"]))]
        sp["hill"] = synth.mabp_hill(a, p, b, c, kT=2.5, stride=stride, w=w)
        out.append(sp)
    return out


def _lookup_tie_steps(spec, s, sb, unit=P.U32):
    """[T] mask of steps whose CV is within the tie band of a half-node:
    4 |u32 - u64| + 1e-6, |u32 - u64| <= unit sb / D (sb: the CVs' rounding
    bounds of the steps, [T, 3])."""
    g = spec["grid"]
    d = len(g["n"])
    D = np.array([(g["hi"][k] - g["lo"][k]) / (g["n"][k] if g["periodic"][k] else g["n"][k] - 1)
                  for k in range(d)])
    u = np.array([P.grid_u(spec, st) for st in s])
    band = 4 * unit * sb[:, :d] / D + 1e-6
    return np.any(np.abs((u % 1.0) - 0.5) < band, axis=1)


def check_mabp(abp, ctx, specs, walkers, Fg, ref, unit=P.U32):
    log = abp.abp_deposit_log_readout(ctx.handle, 1 << 20)
    ids = {w.id: i for i, w in enumerate(walkers)}
    ties = P.compare_deposits(specs, log, ref["deposits"], ids, sb=ref["sb"], unit=unit)
    assert len(ties) <= max(1, len(walkers) // 4), ties
    assert np.all(log["height"] == np.array([specs[ids[int(x)]]["hill"]["w"] for x in log["walker_id"]]))
    off = synth.offsets_of(specs)
    worst = {"V": 0.0, "dV": 0.0, "F": 0.0, "F_step": 0.0, "F_allow": 0.0, "tie_steps": 0}
    for i, (w, sp) in enumerate(zip(walkers, specs)):
        if i in ties:
            continue
        e = P.rel_field_err(ctx.bias(w), ref["fields"][i])
        assert np.all(e < P.TOL_V), (i, e)
        worst["V"] = max(worst["V"], float(e[0]))
        worst["dV"] = max(worst["dV"], float(e[1:].max()))
        keep = ~_lookup_tie_steps(sp, ref["s"][:, i], ref["sb"][:, i], unit)
        worst["tie_steps"] += int((~keep).sum())
        sl = slice(off[i], off[i] + sp["natoms"])
        fe = P.force_err(Fg[keep][:, sl], ref["F"][keep][:, sl])
        assert fe < P.TOL_F, (i, fe)
        worst["F"] = max(worst["F"], float(fe))
        sub = {key: ref[key][keep] for key in ("F", "H", "A", "sb", "Jn")}
        rel, ratio, _ = P.check_forces_per_step(Fg[keep], sub, i, sl, len(sp["grid"]["n"]), unit=unit)
        worst["F_step"] = max(worst["F_step"], rel)
        worst["F_allow"] = max(worst["F_allow"], ratio)
    # the tie band is a few 1e-6 wide in u: a small fraction of steps may fall
    # in it. With uniform fractional parts a step lands there with probability
    # sum_k 2 band_k, so the count is about Poisson with that total as its
    # mean: allow the mean plus four standard deviations (and at least 3, or
    # 0.5 % of the steps)
    lam = 0.0
    for i, sp in enumerate(specs):
        g = sp["grid"]
        d = len(g["n"])
        D = np.array([(g["hi"][k] - g["lo"][k]) / (g["n"][k] if g["periodic"][k] else g["n"][k] - 1)
                      for k in range(d)])
        band = 4 * unit * ref["sb"][:, i, :d] / D + 1e-6
        lam += float(np.minimum(1.0, (2 * band).sum(axis=1)).sum())
    worst["tie_expect"] = lam
    assert worst["tie_steps"] <= max(3, 0.005 * Fg.shape[0] * len(walkers), lam + 4 * np.sqrt(lam) + 3), worst
    return worst


def test_mabp_windowed_two_cv_replay(abp, ctx):
    """COM distance + periodic dihedral walkers with compact hills updated
    every step (the paper's update), dihedral sweeping across +-pi."""
    specs = _mabp(synth.mb64_specs(nw=8, stride=1), a_bins=10.0, c=0.05)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    frames = synth.SweepFrames(8, seed=5, period=(150, 400), dihedral_period=(100, 300)).frames(0, 300)
    Fg = gpu_replay(abp, ctx, walkers, frames, step0=0, chunks=3)
    _, ref = oracle_replay(specs, frames, 0)
    assert np.any(np.abs(np.diff(ref["s"][:, :, 1], axis=0)) > math.pi)
    print("worst", check_mabp(abp, ctx, specs, walkers, Fg, ref))


def test_mabp_chunked_and_single_steps_are_bitwise_equal(abp, ctx):
    specs = _mabp(synth.mb64_specs(nw=4, stride=3), a_bins=8.0, c=0.2)
    frames = synth.SweepFrames(4, seed=8, period=(100, 200)).frames(0, 70)
    wa = ctx.make_walkers(specs)
    Fa = gpu_replay(abp, ctx, wa, frames, 0, chunks=1)
    wb = ctx.make_walkers(specs)
    Fb = gpu_replay(abp, ctx, wb, frames, 0, chunks=9)
    assert np.array_equal(Fa, Fb)
    wc = ctx.make_walkers(specs)
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    F = torch.zeros_like(rec)
    for t in range(frames.shape[0]):
        abp.abp_step(ctx.handle, wc, rec[t], abp.ABP_F32, offs, t)
        abp.abp_forces(ctx.handle, wc, F[t], abp.ABP_F32, offs, abp.ABP_FORCES_OVERWRITE)
    torch.cuda.synchronize()
    assert np.array_equal(F.cpu().numpy()[..., :3].astype(np.float64), Fa)
    for x, y in zip(wa, wc):
        assert np.array_equal(ctx.bias(x), ctx.bias(y))


def test_mabp_per_step_form_with_coordination_numbers(abp, ctx):
    """Walkers with a CN CV run in the per-step fused form (1D, 2D and 3D grids)."""
    specs = _mabp(synth.uneven1000_specs(seed=5, nw=6, stride=2, sizes_2d=(48,), n1d=200, n3d=20), a_bins=4.0,
                  c=0.1, stride=2)
    tm = synth.uneven1000_templates(5, nw=6)
    frames = synth.JitterFrames(tm, seed=6, jitter=0.05).frames(0, 40)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=2)
    _, ref = oracle_replay(specs, frames, 0)
    print("worst", check_mabp(abp, ctx, specs, walkers, Fg, ref))


def test_mabp_plain_form(abp, ctx):
    specs = _mabp(synth.mb64_specs(nw=3, stride=2), a_bins=6.0, c=0.1, stride=2)
    frames = synth.SweepFrames(3, seed=9, period=(100, 200)).frames(0, 30)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    F = torch.zeros_like(rec)
    for t in range(frames.shape[0]):
        abp.abp_step_plain(ctx.handle, walkers, rec[t], abp.ABP_F32, offs, F[t], offs, abp.ABP_FORCES_OVERWRITE, t)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()[..., :3].astype(np.float64)
    _, ref = oracle_replay(specs, frames, 0)
    print("worst", check_mabp(abp, ctx, specs, walkers, Fg, ref))


def test_mabp_fp64_walker(abp, ctx):
    spec = synth.double_well_com_spec()
    spec = _mabp([spec], a_bins=12.0, c=0.05, stride=5)[0]
    x0 = synth.double_well_com_coords(3)
    r = np.random.default_rng(5)
    frames = x0[None] + np.cumsum(r.normal(scale=0.01, size=(80,) + x0.shape), axis=0)
    walkers = ctx.make_walkers([spec], precision=abp.ABP_PREC_FP64)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=2, dtype=np.float64)
    _, ref = oracle_replay([spec], frames, 0)
    print("worst", check_mabp(abp, ctx, [spec], walkers, Fg, ref, unit=P.U64))


def test_rmsd_cvs_on_the_paper_grid(abp, ctx):
    """Two 4-atom RMSD CVs on the 480 x 480 grid over [0, 12] nm, mABP with
    a = 10 grid spacings and p = 20 (the paper's ligand-binding setup), and
    the same CVs with well-tempered Gaussian hills."""
    specs = synth.paper_rmsd_specs(nw=6, c=0.05)
    frames = synth.RmsdFrames(specs, seed=4, period=(400, 1600)).frames(0, 200)  # fast sweeps for coverage
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=2)
    _, ref = oracle_replay(specs, frames, 0)
    assert ref["s"][:, :, :2].min() >= 0.1 and ref["s"][:, :, :2].max() > 1.0
    print("worst mabp", check_mabp(abp, ctx, specs, walkers, Fg, ref))
    wt = []
    for sp in specs:
        sp = dict(sp)
        g = sp["grid"]
        sp["hill"] = synth.hill(0.5, [synth.bins(g, k, 3.0) for k in range(2)], 5, 15.0)
        wt.append(sp)
    ctx2 = abp.Context(0)
    try:
        w2 = ctx2.make_walkers(wt)
        abp.abp_deposit_log_enable(ctx2.handle, 1 << 16)
        Fw = gpu_replay(abp, ctx2, w2, frames, 0)
        _, rw = oracle_replay(wt, frames, 0)
        from tests.test_parity_gpu import check_run

        print("worst wt", check_run(abp, ctx2, wt, w2, frames, 0, Fw, rw))
    finally:
        torch.cuda.synchronize()
        ctx2.close()


def test_mabp_at_the_papers_constants(abp, ctx):
    """b = 0.9, c = 0.001 (the paper's ligand-binding values), compact hills
    a = 10 grid spacings, p = 20, updated every step: the RMSD walkers on the
    paper's 480 x 480 grid (the benchmark's workload) and COM distance +
    dihedral walkers, over 600 steps each."""
    specs = synth.paper_rmsd_specs(nw=6)
    assert all(s["hill"]["b"] == 0.9 and s["hill"]["c"] == 0.001 for s in specs)
    frames = synth.RmsdFrames(specs, seed=5, period=(600, 2400)).frames(0, 600)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=3)
    _, ref = oracle_replay(specs, frames, 0)
    worst = check_mabp(abp, ctx, specs, walkers, Fg, ref)
    print("worst rmsd", worst)
    P.record_errors("paper's RMSD setup, mABP b = 0.9, c = 0.001 (open-loop frames)",
                    "test_mabp_at_the_papers_constants", worst)
    specs2 = _mabp(synth.mb64_specs(nw=6, stride=1), a_bins=10.0, c=0.001, b=0.9)
    frames2 = synth.SweepFrames(6, seed=6, period=(200, 500), dihedral_period=(150, 400)).frames(0, 600)
    ctx2 = abp.Context(0)
    try:
        w2 = ctx2.make_walkers(specs2)
        abp.abp_deposit_log_enable(ctx2.handle, 1 << 16)
        F2 = gpu_replay(abp, ctx2, w2, frames2, 0, chunks=3)
        _, r2 = oracle_replay(specs2, frames2, 0)
        print("worst com/dihedral", check_mabp(abp, ctx2, specs2, w2, F2, r2))
    finally:
        torch.cuda.synchronize()
        ctx2.close()


def test_unsupported_combinations_are_reported(abp, ctx):
    sp = synth.paper_rmsd_specs(nw=1)[0]
    big = dict(sp)
    big["natoms"] = 10
    big["cvs"] = [dict(sp["cvs"][0], a=np.arange(0, 5), ref=np.zeros((5, 3))), sp["cvs"][1]]
    with pytest.raises(abp.AbpError) as e:  # RMSD of 5 atoms: not built
        ctx.make_walkers([big])
    assert e.value.code == abp.ABP_ERR_UNSUPPORTED
    w = ctx.make_walkers([sp])
    rec = torch.zeros(1, 8, 4, device="cuda")
    offs = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(abp.AbpError) as e:  # the plain form has no RMSD
        abp.abp_step_plain(ctx.handle, w, rec[0], abp.ABP_F32, offs, rec[0].clone(), offs, 1, 0)
    assert e.value.code == abp.ABP_ERR_UNSUPPORTED
    shared = _mabp(synth.mb64_specs(nw=1), a_bins=4.0)[0]
    shared["shared"] = "one"
    with pytest.raises(abp.AbpError) as e:  # mABP on a shared grid: not built
        ctx.make_walkers([shared])
    assert e.value.code == abp.ABP_ERR_UNSUPPORTED
    bad = _mabp(synth.mb64_specs(nw=1), a_bins=4.0, b=1.5)[0]
    with pytest.raises(abp.AbpError) as e:
        ctx.make_walkers([bad])
    assert e.value.code == abp.ABP_ERR_INVALID_ARG


def test_range_limit_wall_in_every_form(abp, ctx):
    """The CV range limit (harmonic wall above smax) on the windowed form
    (COM distance + dihedral, WT and mABP) and the per-step form (CN), with
    limits the trajectories cross, against the oracle."""
    specs = synth.mb64_specs(nw=4, stride=5)
    specs = [dict(sp, hill=synth.with_wall(sp["hill"], [1.0, 1.5], 30.0)) for sp in specs]
    specs += [dict(sp, hill=synth.with_wall(sp["hill"], [1.1, 0.0], 10.0))
              for sp in _mabp(synth.mb64_specs(nw=2, stride=2), a_bins=6.0, c=0.1, stride=2)]
    frames = synth.SweepFrames(6, seed=13, period=(100, 200)).frames(0, 120)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=2)
    _, ref = oracle_replay(specs, frames, 0)
    assert np.any(ref["s"][:, :4, 0] > 1.0) and np.any(ref["s"][:, :4, 0] < 1.0)
    off = synth.offsets_of(specs)
    log = abp.abp_deposit_log_readout(ctx.handle, 1 << 20)
    ids = {w.id: i for i, w in enumerate(walkers)}
    ties = P.compare_deposits(specs, log, ref["deposits"], ids, sb=ref["sb"])
    for i, sp in enumerate(specs):
        if i in ties:
            continue
        sl = slice(off[i], off[i] + sp["natoms"])
        keep = ~_lookup_tie_steps(sp, ref["s"][:, i], ref["sb"][:, i]) if i >= 4 else np.ones(len(frames), bool)
        assert P.force_err(Fg[keep][:, sl], ref["F"][keep][:, sl]) < P.TOL_F, i
    cn = [dict(sp, hill=synth.with_wall(sp["hill"], [0.9, 300.0, 300.0][: len(sp["grid"]["n"])], 20.0))
          for sp in synth.uneven1000_specs(seed=7, nw=4, stride=3, sizes_2d=(48,), n1d=200, n3d=20)]
    tm = synth.uneven1000_templates(7, nw=4)
    cframes = synth.JitterFrames(tm, seed=8, jitter=0.05).frames(0, 30)
    ctx2 = abp.Context(0)
    try:
        w2 = ctx2.make_walkers(cn)
        F2 = gpu_replay(abp, ctx2, w2, cframes, 0)
        _, r2 = oracle_replay(cn, cframes, 0)
        assert np.any(r2["dV"] != 0)
        assert P.force_err(F2, r2["F"]) < P.TOL_F
    finally:
        torch.cuda.synchronize()
        ctx2.close()
