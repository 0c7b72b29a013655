"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element. Tolerances: 1e-5 normwise on
V_b and the grid fields; 1e-4 on atom forces, over the run and at every
step (with the FP32 error-model floor of tests/parity.py); CV values of
every deposit within their rounding bound; integer stencil centres
bit-exact outside the FP32 tie band."""
import math

import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import synth
from tests import parity as P

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


def gpu_replay(abp, ctx, walkers, frames, step0, chunks=1, mode=None, init=None, dtype=np.float32):
    """abp_run over frames [T, A, 3] in `chunks` consecutive calls; returns forces [T, A, 3]."""
    mode = abp.ABP_FORCES_OVERWRITE if mode is None else mode
    T, A, _ = frames.shape
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    rec = abp.to_records(frames.astype(dtype), tdt).cuda()
    offs = torch.tensor(synth.offsets_of([w.spec for w in walkers]), dtype=torch.int64, device="cuda")
    F = torch.zeros_like(rec) if init is None else init.clone()
    cdt = abp.ABP_F32 if dtype == np.float32 else abp.ABP_F64
    bounds = np.linspace(0, T, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        abp.abp_run(ctx.handle, walkers, rec[a:], cdt, offs, A, F[a:], offs, A, mode, step0 + a, int(b - a))
    torch.cuda.synchronize()
    return F.cpu().numpy()[..., :3].astype(np.float64)


def oracle_replay(specs, frames, step0, fields=None):
    ws = [oracle.Walker(s) for s in specs]
    return ws, oracle.run(ws, frames.astype(np.float64), synth.offsets_of(specs), step0, frames.shape[0],
                          fields=fields, error_model=True)


def check_run(abp, ctx, specs, walkers, frames, step0, Fg, ref, skip=(), unit=P.U32, log=None):
    """Full comparison: deposits (CV values, centres, heights), grids, forces
    over the run and at every step. Returns the worst figures: grid field
    error, run-normwise force error, per-step force error (relative to the
    step's own force scale), the largest ratio of a step's force error to
    its allowance (tolerance + error-model floor, <= 1) and the number of
    steps that needed the floor."""
    if log is None:
        log = abp.abp_deposit_log_readout(ctx.handle, 1 << 20)
    ids = {w.id: i for i, w in enumerate(walkers)}
    ties = P.compare_deposits(specs, log, ref["deposits"], ids, sb=ref["sb"], unit=unit, step0=step0)
    assert len(ties) <= max(1, len(walkers) // 50), ties
    skip = set(skip) | ties
    off = synth.offsets_of(specs)
    worst = {"V": 0.0, "dV": 0.0, "F": 0.0, "F_step": 0.0, "F_allow": 0.0, "floor_steps": 0}
    for i, (w, sp) in enumerate(zip(walkers, specs)):
        if i in skip:
            continue
        g = ctx.bias(w)
        e = P.rel_field_err(g, ref["fields"][i])
        assert np.all(e < P.TOL_V), (i, e)
        worst["V"] = max(worst["V"], float(e[0]))
        worst["dV"] = max(worst["dV"], float(e[1:].max()))
        sl = slice(off[i], off[i] + sp["natoms"])
        fe = P.force_err(Fg[:, sl], ref["F"][:, sl])
        assert np.all(fe < P.TOL_F), (i, fe.max())
        worst["F"] = max(worst["F"], float(fe.max()))
        rel, ratio, nfloor = P.check_forces_per_step(Fg, ref, i, sl, len(sp["grid"]["n"]), unit=unit)
        worst["F_step"] = max(worst["F_step"], rel)
        worst["F_allow"] = max(worst["F_allow"], ratio)
        worst["floor_steps"] += nfloor
    return worst


# ---------------------------------------------------------------- a1 + a4 + a5 on a given grid


def test_frame_parity_on_uploaded_grid(abp, ctx):
    specs = synth.mb64_specs(nw=6, stride=10 ** 9)
    ws_o = [oracle.Walker(s) for s in specs]
    rng = np.random.default_rng(4)
    fields = []
    for wo in ws_o:
        f = wo.new_field()
        for _ in range(25):
            oracle.deposit(wo, f, [rng.uniform(0.2, 2.0), rng.uniform(-math.pi, math.pi)], rng.uniform(0.1, 1.0))
        fields.append(f)
    walkers = ctx.make_walkers(specs)
    for w, f in zip(walkers, fields):
        ctx.upload_bias(w, f)
        back = ctx.bias(w)
        assert np.abs(back - f).max() <= 1e-14 * np.abs(f).max()
    frames = synth.SweepFrames(6, seed=31).frames(500, 7)
    Fg = gpu_replay(abp, ctx, walkers, frames, step0=1)
    _, ref = oracle_replay(specs, frames, 1, fields=[f.copy() for f in fields])
    off = synth.offsets_of(specs)
    for i, w in enumerate(walkers):
        st = ctx.readout(w)
        np.testing.assert_allclose(st["s"][:2], ref["s"][-1, i, :2], rtol=2e-6, atol=2e-6)
        vmax = np.abs(fields[i][:, 0]).max()
        assert abs(st["V"] - ref["V"][-1, i]) <= P.TOL_V * vmax
        sl = slice(off[i], off[i] + 36)
        assert np.all(P.force_err(Fg[:, sl], ref["F"][:, sl]) < P.TOL_F)


# ---------------------------------------------------------------- open-loop replay with deposits


def test_replay_parity_two_cv_walkers(abp, ctx):
    """COM distance + periodic dihedral walkers (the 64-walker workload's
    shapes), many deposits, the dihedral sweeping across +-pi."""
    specs = synth.mb64_specs(nw=8, stride=5)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    frames = synth.SweepFrames(8, seed=5, period=(150, 400), dihedral_period=(100, 300)).frames(0, 400)
    Fg = gpu_replay(abp, ctx, walkers, frames, step0=0)
    _, ref = oracle_replay(specs, frames, 0)
    worst = check_run(abp, ctx, specs, walkers, frames, 0, Fg, ref)
    print("worst errors", worst)
    P.record_errors("64 walkers, 2 CVs (open-loop frames)", "test_replay_parity_two_cv_walkers", worst)
    # the dihedral did wrap and the deposits did land on both sides of the seam
    assert np.any(np.abs(np.diff(ref["s"][:, :, 1], axis=0)) > math.pi)


def _dihedral_frames(phis, rng):
    """4-atom frames whose IUPAC dihedral is phi by construction."""
    out = []
    for phi in phis:
        x = np.array([[1.0, 0, -0.4], [0, 0, 0], [0, 0, 1.2], [0.7 * math.cos(phi), 0.7 * math.sin(phi), 1.5]])
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(q) < 0:
            q[:, 0] *= -1  # a proper rotation keeps the dihedral's sign
        out.append(x @ q.T * 0.15 + 2.0)
    return np.array(out)[:, :, :]


def test_periodic_seam_hills(abp, ctx):
    """Hills centred within half a spacing of the periodic seam (where the
    centre node wraps to node 0) and exactly on it."""
    n = 64
    D = 2 * math.pi / n
    spec = {"natoms": 4, "cvs": [{"type": "dihedral", "a": [0, 1, 2, 3]}],
            "grid": synth.grid((-math.pi,), (math.pi,), (n,), (True,)),
            "hill": synth.hill(0.7, (0.2,), 1, 10.0)}
    phis = [math.pi - 0.3 * D, math.pi - 0.49 * D, -math.pi + 0.2 * D, math.pi - 1e-4, -math.pi + 0.51 * D,
            math.pi - 0.6 * D, 0.0, math.pi - 0.05 * D]
    frames = _dihedral_frames(phis, np.random.default_rng(3))
    walkers = ctx.make_walkers([spec])
    abp.abp_deposit_log_enable(ctx.handle, 64)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0)
    _, ref = oracle_replay([spec], frames, 0)
    dphi = (ref["s"][:, 0, 0] - np.array(phis) + math.pi) % (2 * math.pi) - math.pi
    assert np.abs(dphi).max() < 1e-5  # FP32 coordinates
    check_run(abp, ctx, [spec], walkers, frames, 0, Fg, ref)


def test_chunked_calls_and_step_forces_are_bitwise_equal(abp, ctx):
    specs = synth.mb64_specs(nw=4, stride=3)
    frames = synth.SweepFrames(4, seed=8, period=(100, 200)).frames(0, 60)
    wa = ctx.make_walkers(specs)
    Fa = gpu_replay(abp, ctx, wa, frames, 0, chunks=1)
    wb = ctx.make_walkers(specs)
    Fb = gpu_replay(abp, ctx, wb, frames, 0, chunks=7)
    assert np.array_equal(Fa, Fb)
    # abp_step + abp_forces, one step per call
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


def test_grid_tile_is_bitwise_exact(abp, ctx):
    """The opt-in shared-memory grid tile (ABP_TUNE_TILE = 1) gives the same
    bits as the untiled path: sweeps that cross the periodic seam and leave
    the tile (forcing reloads), and 1D / 2D / 3D CN walkers. (COM-distance
    and dihedral walkers run in the windowed form, which takes no tile: for
    them the setting must change nothing.)"""
    specs = synth.mb64_specs(nw=6, stride=4)
    frames = synth.SweepFrames(6, seed=18, period=(60, 90), dihedral_period=(40, 70)).frames(0, 240)
    w0 = ctx.make_walkers(specs)
    F0 = gpu_replay(abp, ctx, w0, frames, 0, chunks=4)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TILE, 1)
    w1 = ctx.make_walkers(specs)
    F1 = gpu_replay(abp, ctx, w1, frames, 0, chunks=4)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TILE, -1)
    assert np.array_equal(F0, F1)
    for a, b in zip(w0, w1):
        assert np.array_equal(ctx.bias(a), ctx.bias(b))
    uspecs = synth.uneven1000_specs(seed=5, nw=6, stride=6, sizes_2d=(48,), n1d=200, n3d=20)
    tm = synth.uneven1000_templates(5, nw=6)
    uframes = synth.JitterFrames(tm, seed=6, jitter=0.05).frames(0, 48)
    u0 = ctx.make_walkers(uspecs)
    G0 = gpu_replay(abp, ctx, u0, uframes, 0, chunks=2)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TILE, 1)
    u1 = ctx.make_walkers(uspecs)
    G1 = gpu_replay(abp, ctx, u1, uframes, 0, chunks=2)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TILE, -1)
    assert np.array_equal(G0, G1)
    for a, b in zip(u0, u1):
        assert np.array_equal(ctx.bias(a), ctx.bias(b))


def test_lean_instantiation_matches(abp, ctx):
    """The 128-register instantiation (ABP_TUNE_LEAN) computes the same steps:
    CN walkers of the uneven mix, group width fixed."""
    specs = synth.uneven1000_specs(seed=8, nw=8, stride=5, sizes_2d=(48,), n1d=200, n3d=20)
    tm = synth.uneven1000_templates(8, nw=8)
    frames = synth.JitterFrames(tm, seed=9).frames(0, 20)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUP_THREADS, 64)
    w0 = ctx.make_walkers(specs)
    F0 = gpu_replay(abp, ctx, w0, frames, 0)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_LEAN, 1)
    w1 = ctx.make_walkers(specs)
    F1 = gpu_replay(abp, ctx, w1, frames, 0)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_LEAN, 0)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUP_THREADS, 0)
    assert P.force_err(F1, F0) < 1e-6
    for a, b in zip(w0, w1):
        assert np.all(P.rel_field_err(ctx.bias(b), ctx.bias(a)) < 1e-7)
    print("lean bitwise equal:", np.array_equal(F0, F1))


def test_plain_form_matches_batched_and_oracle(abp, ctx):
    specs = synth.mb64_specs(nw=3, stride=4)
    frames = synth.SweepFrames(3, seed=9, period=(100, 200)).frames(0, 40)
    wa = ctx.make_walkers(specs)
    Fa = gpu_replay(abp, ctx, wa, frames, 0)
    wp = ctx.make_walkers(specs)
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    F = torch.zeros_like(rec)
    for t in range(frames.shape[0]):
        abp.abp_step_plain(ctx.handle, wp, rec[t], abp.ABP_F32, offs, F[t], offs, abp.ABP_FORCES_OVERWRITE, t)
    torch.cuda.synchronize()
    Fp = F.cpu().numpy()[..., :3].astype(np.float64)
    _, ref = oracle_replay(specs, frames, 0)
    off = synth.offsets_of(specs)
    for i in range(3):
        sl = slice(off[i], off[i] + 36)
        assert np.all(P.force_err(Fp[:, sl], ref["F"][:, sl]) < P.TOL_F)
        assert np.all(P.force_err(Fp[:, sl], Fa[:, sl]) < P.TOL_F)
        assert np.all(P.rel_field_err(ctx.bias(wp[i]), ref["fields"][i]) < P.TOL_V)


def test_batch_invariance_bitwise(abp, ctx):
    """A walker's result is bit-identical alone and inside a larger batch
    (same launch shape): per-walker reductions have a fixed order."""
    specs = synth.mb64_specs(nw=12, stride=5)
    frames = synth.SweepFrames(12, seed=10, period=(200, 300)).frames(0, 50)
    wall = ctx.make_walkers(specs)
    Fall = gpu_replay(abp, ctx, wall, frames, 0)
    off = synth.offsets_of(specs)
    for i in (0, 5, 11):
        w1 = ctx.make_walkers([specs[i]])
        fr = frames[:, off[i]:off[i] + 36]
        F1 = gpu_replay(abp, ctx, w1, fr, 0)
        assert np.array_equal(F1, Fall[:, off[i]:off[i] + 36])
        assert np.array_equal(ctx.bias(w1[0]), ctx.bias(wall[i]))


# ---------------------------------------------------------------- uneven batch with CN


def test_uneven_batch_with_coordination_numbers(abp, ctx):
    """1D / 2D / 3D walkers with a 40 x 400 coordination number (the uneven
    workload's CV mix) on reduced grid sizes, in one launch."""
    nw = 20
    specs = synth.uneven1000_specs(seed=3, nw=nw, stride=10, sizes_2d=(48, 64), n1d=256, n3d=24)
    tm = synth.uneven1000_templates(3, nw=nw)
    # the CN axis range holds the templates' CN
    for sp, t in zip(specs, tm):
        wo = oracle.Walker(sp)
        cn = oracle.cv_eval(wo, len(sp["cvs"]) - 1, t)[0]
        assert synth.CN_RANGE_UNEVEN[0] + 20 < cn < synth.CN_RANGE_UNEVEN[1] - 20
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    frames = synth.JitterFrames(tm, seed=4).frames(0, 60)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0)
    _, ref = oracle_replay(specs, frames, 0)
    worst = check_run(abp, ctx, specs, walkers, frames, 0, Fg, ref)
    print("worst errors", worst)
    assert {len(s["grid"]["n"]) for s in specs} == {1, 2, 3}


def test_uneven_batch_full_size_autotuned_launch(abp, ctx):
    """250 walkers of the uneven workload with its real grids (1D 1024
    nodes; 2D 128^2, 256^2, 512^2; 3D 64^3; CN 40 x 400) and its deposit
    stride, in launches of the shape the autotuner picks for them (as the
    benchmark runs them), every walker compared with the oracle element by
    element over 150 steps (three deposits each)."""
    from paper_1609_09833_gb300 import autotune

    nw, T, C = 250, 150, 25
    specs = synth.uneven1000_specs(seed=31, nw=nw)
    assert {tuple(s["grid"]["n"]) for s in specs} >= {(1024,), (128, 128), (256, 256), (512, 512), (64, 64, 64)}
    tm = synth.uneven1000_templates(31, nw=nw)
    frames = synth.JitterFrames(tm, seed=32).frames(0, T)
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    tuned = autotune.tune(ctx, specs, rec, offs, C, cache_path=None)["best"]
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=T // C)
    _, ref = oracle_replay(specs, frames, 0)
    worst = check_run(abp, ctx, specs, walkers, frames, 0, Fg, ref)
    print("launch shape", tuned, "worst errors", worst)
    P.record_errors("uneven 1000 walkers (250 at full size, autotuned launch)",
                    "test_uneven_batch_full_size_autotuned_launch", worst)


# ---------------------------------------------------------------- FP64 end to end


def test_fp64_single_walker(abp, ctx):
    """The double-well COM walker in FP64 end to end: agreement to ~1e-10."""
    spec = synth.double_well_com_spec(stride=7)
    x0 = synth.double_well_com_coords(21)
    rng = np.random.default_rng(22)
    T = 300
    steps = rng.normal(scale=0.03, size=(T, 16, 3))
    frames = x0[None] + np.cumsum(steps, axis=0)
    walkers = ctx.make_walkers([spec], precision=1)
    abp.abp_deposit_log_enable(ctx.handle, 4096)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, dtype=np.float64)
    _, ref = oracle_replay([spec], frames, 0)
    g = ctx.bias(walkers[0])
    e = P.rel_field_err(g, ref["fields"][0])
    assert np.all(e < 1e-10)
    fe = P.force_err(Fg, ref["F"])
    assert np.all(fe < 1e-9)
    rel, ratio, nfloor = P.check_forces_per_step(Fg, ref, 0, slice(0, 16), 1, tol=1e-9, unit=P.U64)
    print("per step", rel, ratio, nfloor)
    P.record_errors("1 walker FP64, double well (open-loop frames)", "test_fp64_single_walker",
                    {"V": e[0], "dV": e[1:].max(), "F": fe, "F_step": rel, "F_allow": ratio, "floor_steps": nfloor})
    log = abp.abp_deposit_log_readout(ctx.handle, 4096)
    np.testing.assert_array_equal(log["ic"][:, 0], ref["deposits"]["ic"][:, 0])
    np.testing.assert_allclose(log["height"], ref["deposits"]["height"], rtol=1e-12)


# ---------------------------------------------------------------- modes and edge cases


def test_accumulate_mode_adds_to_caller_forces(abp, ctx):
    specs = synth.mb64_specs(nw=2, stride=2)
    frames = synth.SweepFrames(2, seed=12).frames(0, 6)
    w1 = ctx.make_walkers(specs)
    F1 = gpu_replay(abp, ctx, w1, frames, 0)
    w2 = ctx.make_walkers(specs)
    base = torch.randn(frames.shape[0], frames.shape[1], 4, device="cuda")
    F2 = gpu_replay(abp, ctx, w2, frames, 0, mode=abp.ABP_FORCES_ACCUMULATE, init=base)
    b = base.cpu().numpy()[..., :3].astype(np.float64)
    np.testing.assert_allclose(F2, F1 + b, rtol=1e-6, atol=1e-6)


def test_out_of_range_cv_is_clamped_and_clipped(abp, ctx):
    specs = synth.mb64_specs(nw=2, stride=3)
    for sp in specs:
        sp["grid"] = synth.grid((0.2, -math.pi), (0.9, math.pi), (200, 128), (False, True))
    frames = synth.SweepFrames(2, seed=13, r_range=(0.5, 1.4), period=(60, 80)).frames(0, 90)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 4096)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0)
    _, ref = oracle_replay(specs, frames, 0)
    assert np.any(ref["flags"] & oracle.FLAG_OOR)
    check_run(abp, ctx, specs, walkers, frames, 0, Fg, ref)
    st = ctx.readout(walkers[0])
    assert bool(st["flags"] & abp.WFLAG_OOR) == bool(ref["flags"][-1, 0] & oracle.FLAG_OOR)


def test_nonfinite_coordinates_leave_state_unchanged(abp, ctx):
    specs = synth.mb64_specs(nw=2, stride=1)
    walkers = ctx.make_walkers(specs)
    frames = synth.SweepFrames(2, seed=14).frames(0, 1)
    frames[0, 3, 1] = np.nan  # walker 0
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor([0, 36], dtype=torch.int64, device="cuda")
    F = torch.full_like(rec, 7.0)
    abp.abp_run(ctx.handle, walkers, rec, abp.ABP_F32, offs, 72, F, offs, 72, abp.ABP_FORCES_OVERWRITE, 0, 1)
    with pytest.raises(abp.AbpError) as e:
        abp.abp_sync(ctx.handle)
    assert e.value.code == abp.ABP_ERR_NONFINITE
    abp.abp_sync(ctx.handle)  # the counter was reset
    assert np.all(ctx.bias(walkers[0]) == 0.0)
    assert np.any(ctx.bias(walkers[1]) != 0.0)
    assert torch.all(F[0, :36, :3] == 0)
    st = ctx.readout(walkers[0])
    assert st["status"] == abp.ABP_ERR_NONFINITE and st["flags"] == abp.WFLAG_NONFINITE


def test_empty_and_zero_step_calls(abp, ctx):
    specs = synth.mb64_specs(nw=1, stride=1)
    walkers = ctx.make_walkers(specs)
    abp.abp_run(ctx.handle, [], None, abp.ABP_F32, None, 0, None, None, 0, 0, 0, 1)
    rec = torch.zeros(1, 36, 4, device="cuda")
    offs = torch.zeros(1, dtype=torch.int64, device="cuda")
    abp.abp_run(ctx.handle, walkers, rec, abp.ABP_F32, offs, 36, rec, offs, 36, 1, 0, 0)
    abp.abp_sync(ctx.handle)
    assert np.all(ctx.bias(walkers[0]) == 0.0)


def test_invalid_arguments_are_reported(abp, ctx):
    specs = synth.mb64_specs(nw=2, stride=1)
    walkers = ctx.make_walkers(specs)
    rec = torch.zeros(2, 72, 4, device="cuda")
    offs = torch.tensor([0, 36], dtype=torch.int64, device="cuda")
    with pytest.raises(abp.AbpError) as e:  # dtype mismatch
        abp.abp_run(ctx.handle, walkers, rec, abp.ABP_F64, offs, 72, rec, offs, 72, 1, 0, 1)
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    raw = torch.zeros(2 * 72 * 4 + 1, device="cuda")
    with pytest.raises(abp.AbpError) as e:  # misaligned coordinates
        abp.abp_run(ctx.handle, walkers, raw.data_ptr() + 4, abp.ABP_F32, offs, 72, rec, offs, 72, 1, 0, 1)
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    with pytest.raises(abp.AbpError) as e:  # FP64 walker mixed with FP32 walkers
        w64 = ctx.make_walkers([synth.double_well_com_spec()], precision=1)
        abp.abp_run(ctx.handle, walkers + w64, rec, abp.ABP_F32, offs, 72, rec, offs, 72, 1, 0, 1)
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    with pytest.raises(abp.AbpError) as e:  # a periodic stencil wider than its axis
        bad = dict(specs[0])
        bad["grid"] = synth.grid((0.2, -math.pi), (2.0, math.pi), (64, 16), (False, True))
        bad["hill"] = dict(specs[0]["hill"], sigma=[0.04, 1.0])
        ctx.make_walkers([bad])
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    with pytest.raises(abp.AbpError) as e:  # duplicate atom in a group
        bad = dict(specs[0])
        bad["cvs"] = [{"type": "com_dist", "a": [0, 0, 1], "b": [2, 3]}, specs[0]["cvs"][1]]
        ctx.make_walkers([bad])
    assert e.value.code == abp.ABP_ERR_INVALID_ARG


def test_hbm_budget_admission(abp):
    c = abp.Context(0, budget=64 << 20)
    try:
        specs = synth.mb64_specs(nw=40)  # 2 MB of grid per walker
        with pytest.raises(abp.AbpError) as e:
            c.make_walkers(specs)
        assert e.value.code == abp.ABP_ERR_ADMISSION
        used, budget = abp.abp_ctx_bytes(c.handle)
        assert used <= budget
    finally:
        c.close()


# ---------------------------------------------------------------- full-size workload, sampled


def test_full_size_64_walker_workload_sampled(abp, ctx):
    """64 walkers with their own 256 x 256 grids, chunked launches as the
    benchmark runs them; six walkers (sampled by seed) checked against the
    oracle."""
    nw, T = 64, 300
    specs = synth.mb64_specs(nw=nw)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    fr = synth.SweepFrames(nw, seed=77)
    frames = fr.frames(0, T)
    Fg = gpu_replay(abp, ctx, walkers, frames, 0, chunks=3)
    pick = sorted(np.random.default_rng(78).choice(nw, 6, replace=False))
    off = synth.offsets_of(specs)
    sub = [specs[i] for i in pick]
    subframes = np.concatenate([frames[:, off[i]:off[i] + 36] for i in pick], axis=1)
    _, ref = oracle_replay(sub, subframes, 0)
    log = abp.abp_deposit_log_readout(ctx.handle, 1 << 16)
    assert log["total"] == nw * (T // 50)
    Fsub = np.concatenate([Fg[:, off[i]:off[i] + 36] for i in pick], axis=1)
    for j, i in enumerate(pick):
        assert np.all(P.rel_field_err(ctx.bias(walkers[i]), ref["fields"][j]) < P.TOL_V)
        fe = P.force_err(Fg[:, off[i]:off[i] + 36], ref["F"][:, j * 36:(j + 1) * 36])
        assert np.all(fe < P.TOL_F)
        P.check_forces_per_step(Fsub, ref, j, slice(j * 36, (j + 1) * 36), 2)


def test_all_steps_accumulated_into_one_force_buffer(abp, ctx):
    """force_step_stride = 0 with ACCUMULATE: every step's force is added to
    the same records, in step order (windowed form and per-step form)."""
    for specs, frames in ((synth.mb64_specs(nw=3, stride=4), synth.SweepFrames(3, seed=14).frames(0, 45)),
                          (synth.uneven1000_specs(seed=9, nw=3, stride=4, sizes_2d=(48,), n1d=200, n3d=20),
                           synth.JitterFrames(synth.uneven1000_templates(9, nw=3), seed=10).frames(0, 12))):
        wa = ctx.make_walkers(specs)
        Fa = gpu_replay(abp, ctx, wa, frames, 0)  # one force record set per step
        wb = ctx.make_walkers(specs)
        rec = abp.to_records(frames).cuda()
        A = rec.shape[1]
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        base = torch.randn(A, 4, device="cuda")
        F = base.clone()
        abp.abp_run(ctx.handle, wb, rec, abp.ABP_F32, offs, A, F, offs, 0, abp.ABP_FORCES_ACCUMULATE, 0,
                    frames.shape[0])
        torch.cuda.synchronize()
        want = base.cpu().numpy()[:, :3].astype(np.float64) + Fa.sum(axis=0)
        np.testing.assert_allclose(F.cpu().numpy()[:, :3], want, rtol=1e-5, atol=1e-5 * np.abs(Fa).max())
        for x, y in zip(wa, wb):
            assert np.array_equal(ctx.bias(x), ctx.bias(y))


def test_checkpoint_and_resume_is_bit_exact(abp, ctx):
    """Save a walker's grid after step k (abp_grid_save), restore it into a
    new walker (abp_grid_restore) and continue: the forces and the grid equal
    an uninterrupted run bit for bit (a walker on its own grid; windowed and
    per-step forms, mABP and WT). Through FP64 values (abp_bias_readout /
    abp_bias_upload) the resumed run agrees to rounding."""
    cases = (synth.mb64_specs(nw=2, stride=3),
             [dict(sp, hill=synth.mabp_hill([synth.bins(sp["grid"], k, 6.0) for k in range(2)], 20, 0.9, 0.2,
                                            stride=2)) for sp in synth.mb64_specs(nw=2)],
             synth.uneven1000_specs(seed=4, nw=2, stride=3, sizes_2d=(48,), n1d=200, n3d=20))
    for specs in cases:
        if specs[0]["cvs"][-1]["type"] == "coord":
            frames = synth.JitterFrames(synth.uneven1000_templates(4, nw=2), seed=5).frames(0, 30)
        else:
            frames = synth.SweepFrames(2, seed=15).frames(0, 30)
        wa = ctx.make_walkers(specs)
        Fa = gpu_replay(abp, ctx, wa, frames, 0)
        k = 17
        wb = ctx.make_walkers(specs)
        gpu_replay(abp, ctx, wb, frames[:k], 0)
        saved = [abp.abp_grid_save(ctx.handle, w.grid) for w in wb]
        values = [ctx.bias(w) for w in wb]
        wc = ctx.make_walkers(specs)
        for w, g in zip(wc, saved):
            abp.abp_grid_restore(ctx.handle, w.grid, g)
        wv = ctx.make_walkers(specs)
        for w, g in zip(wv, values):
            ctx.upload_bias(w, g)
        rec = abp.to_records(frames[k:]).cuda()
        A = rec.shape[1]
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        F = torch.zeros_like(rec)
        Fv = torch.zeros_like(rec)
        abp.abp_run(ctx.handle, wc, rec, abp.ABP_F32, offs, A, F, offs, A, abp.ABP_FORCES_OVERWRITE, k,
                    frames.shape[0] - k)
        abp.abp_run(ctx.handle, wv, rec, abp.ABP_F32, offs, A, Fv, offs, A, abp.ABP_FORCES_OVERWRITE, k,
                    frames.shape[0] - k)
        torch.cuda.synchronize()
        assert np.array_equal(F.cpu().numpy()[..., :3].astype(np.float64), Fa[k:])
        for x, y in zip(wa, wc):
            assert np.array_equal(ctx.bias(x), ctx.bias(y))
        assert P.force_err(Fv.cpu().numpy()[..., :3].astype(np.float64), Fa[k:]) < 1e-6


@pytest.mark.parametrize("kind", ["wt", "mabp", "fp64"])
def test_windowed_launch_shapes_give_the_same_bits(abp, ctx, kind):
    """The windowed form's result does not depend on its launch shape: one
    256-thread group per CTA (CV and chain halves decoupled by named
    barriers), two 128-thread groups per CTA (lockstep halves), 64-thread
    groups and one-warp groups (the three phases in turn) give the same
    forces and grids, over calls of several windows."""
    from tests.test_mabp_gpu import _mabp

    dtype = np.float32
    if kind == "fp64":
        specs = [synth.double_well_com_spec(stride=7)] * 3
        x0 = synth.double_well_com_coords(5)
        frames = x0[None] + np.cumsum(synth.rng(6).normal(scale=0.03, size=(150, 16, 3)), axis=0)
        frames = np.concatenate([frames + 0.1 * i for i in range(3)], axis=1)
        dtype = np.float64
    else:
        specs = synth.mb64_specs(nw=4, stride=9)
        if kind == "mabp":
            specs = _mabp(specs, a_bins=8.0, c=0.2, stride=3)
        frames = synth.SweepFrames(4, seed=12, period=(100, 200)).frames(0, 150)
    runs = []
    for G, gpc in ((256, 1), (128, 2), (64, 1), (32, 4)):
        abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUP_THREADS, G)
        abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUPS_PER_CTA, gpc)
        prec = abp.ABP_PREC_FP64 if kind == "fp64" else abp.ABP_PREC_FP32_COMP
        w = ctx.make_walkers(specs, precision=prec)
        F = gpu_replay(abp, ctx, w, frames, 0, chunks=2, dtype=dtype)
        runs.append((G, gpc, F, [ctx.bias(x) for x in w]))
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUP_THREADS, 0)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUPS_PER_CTA, 0)
    G0, p0, F0, B0 = runs[0]
    assert np.count_nonzero(F0) > 0
    for G, gpc, F, B in runs[1:]:
        assert np.array_equal(F, F0), (G, gpc, np.argwhere(F != F0)[:3])
        for a, b in zip(B, B0):
            assert np.array_equal(a, b), (G, gpc)
