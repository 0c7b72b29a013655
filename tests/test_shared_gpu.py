"""GPU parity of the phased form: walkers sharing one grid (multiple-walker
runs, FP64 accumulator shadow, Jacobi order within a step) and walkers too
large for one shared-memory walker group, against the FP64 oracle run with
one shared field (the oracle applies the step's hills in walker order; the
GPU adds them with FP64 atomics, so the two agree up to FP64 rounding)."""
import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import synth
from tests import parity as P
from tests.test_parity_gpu import check_run, gpu_replay

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


def _shared_oracle(specs, frames, step0):
    ws = [oracle.Walker(s) for s in specs]
    shared = ws[0].new_field()
    return oracle.run(ws, frames.astype(np.float64), synth.offsets_of(specs), step0, frames.shape[0],
                      fields=[shared] * len(ws), error_model=True)


def test_shared_grid_small(abp, ctx):
    """Six walkers (COM distance, dihedral, CN over 20 x 300 atoms in a 3 nm
    periodic box) depositing into one 40^3 grid every second step."""
    nw = 6
    specs = synth.shared256_specs(nw=nw, n=40, n_lig=20, n_env=300, box=3.0, stride=2, cn_range=(60.0, 160.0))
    tm = synth.shared256_templates(9, nw=nw, n_lig=20, n_env=300, box=3.0)
    frames = synth.JitterFrames(tm, seed=10, jitter=0.01).frames(0, 9)
    walkers = ctx.make_walkers(specs)
    assert len({w.grid for w in walkers}) == 1
    abp.abp_deposit_log_enable(ctx.handle, 4096)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=2)
    ref = _shared_oracle(specs, frames, 0)
    assert len(ref["deposits"]["step"]) == nw * 5
    # every walker's view of the one grid is the same grid: compare it once
    worst = check_run(abp, ctx, specs, walkers, frames, 0, Fg, ref)
    print("worst errors", worst)


def test_shared_grid_single_step_calls(abp, ctx):
    """abp_step + abp_forces on a shared grid equal one multi-step abp_run."""
    nw = 4
    specs = synth.shared256_specs(nw=nw, n=32, n_lig=16, n_env=200, box=3.0, stride=1, cn_range=(30.0, 130.0))
    tm = synth.shared256_templates(11, nw=nw, n_lig=16, n_env=200, box=3.0)
    frames = synth.JitterFrames(tm, seed=12, jitter=0.01).frames(0, 4)
    wa = ctx.make_walkers(specs)
    Fa = gpu_replay(abp, ctx, wa, frames, 0)
    for sp in specs:
        sp["shared"] = "second"
    wb = ctx.make_walkers(specs)
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    F = torch.zeros_like(rec)
    for t in range(frames.shape[0]):
        abp.abp_step(ctx.handle, wb, rec[t], abp.ABP_F32, offs, t)
        abp.abp_forces(ctx.handle, wb, F[t], abp.ABP_F32, offs, abp.ABP_FORCES_OVERWRITE)
    torch.cuda.synchronize()
    Fb = F.cpu().numpy()[..., :3].astype(np.float64)
    # FP64 atomics may add the step's hills in another order: agreement to rounding
    assert P.force_err(Fb, Fa) < 1e-6
    assert np.all(P.rel_field_err(ctx.bias(wb[0]), ctx.bias(wa[0])) < 1e-9)


def test_large_walker_on_own_grid(abp, ctx):
    """A walker whose CN covers 64 x 9000 atoms (too many atoms for one
    shared-memory walker group) runs in the phased form on its own grid."""
    n_lig, n_env = 64, 9000
    spec = synth.shared256_specs(nw=1, n=48, n_lig=n_lig, n_env=n_env, box=6.0, stride=3, cn_range=(1000.0, 1500.0))[0]
    spec.pop("shared")
    tm = synth.shared256_templates(13, nw=1, n_lig=n_lig, n_env=n_env, box=6.0)
    wo = oracle.Walker(spec)
    cn = oracle.cv_eval(wo, 2, tm[0])[0]
    assert 1050 < cn < 1450, cn
    frames = synth.JitterFrames(tm, seed=14, jitter=0.01).frames(0, 7)
    walkers = ctx.make_walkers([spec])
    abp.abp_deposit_log_enable(ctx.handle, 4096)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0)
    ref = oracle.run([wo], frames.astype(np.float64), [0], 0, frames.shape[0], error_model=True)
    print("worst errors", check_run(abp, ctx, [spec], walkers, frames, 0, Fg, ref))
    with pytest.raises(abp.AbpError):  # the plain form does not take it
        rec = abp.to_records(frames[:1]).cuda()
        offs = torch.zeros(1, dtype=torch.int64, device="cuda")
        abp.abp_step_plain(ctx.handle, walkers, rec[0], abp.ABP_F32, offs, rec[0].clone(), offs, 1, 0)


def test_walkers_on_one_unshared_grid_are_rejected(abp, ctx):
    specs = synth.mb64_specs(nw=2)
    g = ctx.make_grid(specs[0]["grid"])
    hs = []
    for sp in specs:
        desc, keep = abp.walker_desc(sp)
        hs.append(abp.abp_walker_create(ctx.handle, g, desc))
    rec = torch.zeros(1, 72, 4, device="cuda")
    offs = torch.tensor([0, 36], dtype=torch.int64, device="cuda")
    with pytest.raises(abp.AbpError) as e:
        abp.abp_run(ctx.handle, hs, rec, abp.ABP_F32, offs, 72, rec.clone(), offs, 72, 1, 0, 1)
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    for h in hs:
        abp.abp_walker_destroy(h)


def test_full_size_shared_256_workload(abp, ctx):
    """32 walkers, 200 ligand + 10,000 environment atoms each in a 6 nm
    periodic box, one shared 256^3 grid, deposit every 10 steps: three steps
    (one deposit step of all 32 walkers) checked against the oracle run at
    full size."""
    nw = 32
    specs = synth.shared256_specs(nw=nw)
    tm = synth.shared256_templates(21, nw=nw)
    frames = synth.JitterFrames(tm, seed=22).frames(0, 3)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 4096)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0)
    ref = _shared_oracle(specs, frames, 0)
    assert np.all((ref["s"][0, :, 2] > synth.CN_RANGE_SHARED[0]) & (ref["s"][0, :, 2] < synth.CN_RANGE_SHARED[1]))
    log = abp.abp_deposit_log_readout(ctx.handle, 4096)
    assert log["total"] == nw
    np.testing.assert_allclose(log["height"], 0.2, rtol=1e-12)  # an empty grid: every hill has height w
    g = ctx.bias(walkers[0])
    e = P.rel_field_err(g, ref["fields"][0])
    assert np.all(e < P.TOL_V)
    off = synth.offsets_of(specs)
    ids = {w.id: i for i, w in enumerate(walkers)}
    assert not P.compare_deposits(specs, log, ref["deposits"], ids, sb=ref["sb"])
    worst = {"V": e[0], "dV": e[1:].max(), "F": 0.0, "F_step": 0.0, "F_allow": 0.0, "floor_steps": 0}
    for i in range(nw):
        sl = slice(off[i], off[i] + specs[i]["natoms"])
        fe = P.force_err(Fg[:, sl], ref["F"][:, sl])
        assert fe < P.TOL_F
        rel, ratio, nfloor = P.check_forces_per_step(Fg, ref, i, sl, 3)
        worst["F"] = max(worst["F"], fe)
        worst["F_step"] = max(worst["F_step"], rel)
        worst["F_allow"] = max(worst["F_allow"], ratio)
        worst["floor_steps"] += nfloor
    print("worst errors", worst)
    P.record_errors("shared 256^3, 32 walkers (open-loop frames, full size)", "test_full_size_shared_256_workload",
                    worst)


def test_cuda_graph_replay_equals_direct_calls(abp, ctx):
    """abp_run captured in a CUDA graph (after one direct call has cached the
    walker tables) gives the same results as direct calls: bit for bit in the
    fused form, to FP64 rounding on a shared grid."""
    specs = synth.mb64_specs(nw=4, stride=3)
    frames = synth.SweepFrames(4, seed=51).frames(0, 12)
    rec = abp.to_records(frames).cuda()
    A = rec.shape[1]
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    wa = ctx.make_walkers(specs)
    Fa = torch.zeros_like(rec)
    for c in range(3):  # three calls of 4 steps
        abp.abp_run(ctx.handle, wa, rec[4 * c:], abp.ABP_F32, offs, A, Fa[4 * c:], offs, A, 1, 4 * c, 4)
    wb = ctx.make_walkers(specs)
    Fb = torch.zeros_like(rec)
    abp.abp_run(ctx.handle, wb, rec, abp.ABP_F32, offs, A, Fb, offs, A, 1, 0, 4)  # direct: tables cached
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    ctx.set_stream(s.cuda_stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        abp.abp_run(ctx.handle, wb, rec[4:], abp.ABP_F32, offs, A, Fb[4:], offs, A, 1, 4, 4)
    g.replay()
    torch.cuda.synchronize()
    ctx.set_stream(torch.cuda.current_stream().cuda_stream)
    # the graph holds steps 4..7; replaying it again would re-apply them, so
    # run steps 8..11 directly and compare everything
    abp.abp_run(ctx.handle, wb, rec[8:], abp.ABP_F32, offs, A, Fb[8:], offs, A, 1, 8, 4)
    torch.cuda.synchronize()
    assert torch.equal(Fa, Fb)
    for x, y in zip(wa, wb):
        assert np.array_equal(ctx.bias(x), ctx.bias(y))
