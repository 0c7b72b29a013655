"""GPU parity of the closed-loop form (abp_md_run): the force call inside the
model MD engine, step t + 1's coordinates from step t's bias force on the
device.

Against the oracle, one step at a time along the oracle's own closed-loop
trajectory (the oracle's coordinates go in; nothing of the GPU's goes into
the oracle): at every step the GPU's bias force, deposits and grid meet
the open-loop tolerances, and its move lands where the oracle's did within
the FP32 (or FP64) error of one move. Then the GPU's own closed loop:
launches of many steps equal one-step calls bit for bit; the open-loop
windowed form replayed on the GPU's own trajectory gives the same forces
and grid; and the bias converges to the well-tempered limit of the
COM-distance double well, -(1 - 1/gamma) (U(s) - 2 kT ln s) + C."""
import math

import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import synth
from tests import parity as P
from tests.test_parity_gpu import check_run, gpu_replay, oracle_replay

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


def _tdt(dtype):
    return torch.float32 if dtype == np.float32 else torch.float64


def gpu_steps_from(abp, ctx, walkers, frames, md, streams, step0=0, dtype=np.float32):
    """One closed-loop call per step, each starting from frames[t] (the
    oracle's trajectory): returns the moved coordinates and the bias forces,
    [T, atoms, 3] each."""
    specs = [w.spec for w in walkers]
    rec = abp.to_records(frames.astype(dtype), _tdt(dtype)).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    cdt = abp.ABP_F32 if dtype == np.float32 else abp.ABP_F64
    X = torch.zeros_like(rec)
    F = torch.zeros_like(rec)
    buf = torch.zeros_like(rec[0])
    for t in range(frames.shape[0]):
        buf.copy_(rec[t])
        abp.abp_md_run(ctx.handle, walkers, buf, cdt, offs, md, streams, forces=F[t], force_offsets=offs,
                       mode=abp.ABP_FORCES_OVERWRITE, step0=step0 + t, nsteps=1)
        X[t].copy_(buf)
    torch.cuda.synchronize()
    return X.cpu().numpy()[..., :3].astype(np.float64), F.cpu().numpy()[..., :3].astype(np.float64)


def gpu_run(abp, ctx, walkers, x0, md, streams, step0, nsteps, chunks=1, dtype=np.float32):
    """The GPU's own closed loop from x0 in `chunks` calls: returns the
    trajectory (coordinates each step was evaluated at), the bias forces and
    the final coordinates."""
    specs = [w.spec for w in walkers]
    A = x0.shape[0]
    tdt = _tdt(dtype)
    buf = abp.to_records(x0[None].astype(dtype), tdt).cuda()[0]
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    cdt = abp.ABP_F32 if dtype == np.float32 else abp.ABP_F64
    traj = torch.zeros(nsteps, A, 4, dtype=tdt, device="cuda")
    F = torch.zeros_like(traj)
    bounds = np.linspace(0, nsteps, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        abp.abp_md_run(ctx.handle, walkers, buf, cdt, offs, md, streams, traj=traj[a:], traj_offsets=offs,
                       traj_step_stride=A, forces=F[a:], force_offsets=offs, force_step_stride=A,
                       mode=abp.ABP_FORCES_OVERWRITE, step0=step0 + a, nsteps=int(b - a))
    torch.cuda.synchronize()
    cv = lambda t: t.cpu().numpy()[..., :3].astype(np.float64)  # noqa: E731
    return cv(traj), cv(F), cv(buf)


def _potential_floor(md, ref, sl, w, d, unit):
    """Per step and atom, the error the FP32 (FP64) CV potential's force may
    carry: its slope (central differences of dU/ds) times the CVs' rounding
    bounds, plus its own rounding; and a bound on the force's size."""
    T = ref["s"].shape[0]
    E = np.zeros((T, d))
    G = np.zeros((T, d))
    for t in range(T):
        s = ref["s"][t, w, :d]
        _, dU = oracle.md_potential(md, s)
        G[t] = np.abs(dU[:d])
        H = np.zeros((d, d))
        for j in range(d):
            e = 1e-6 * max(1.0, abs(s[j]))
            sp, sm = s.copy(), s.copy()
            sp[j] += e
            sm[j] -= e
            H[:, j] = (oracle.md_potential(md, sp)[1][:d] - oracle.md_potential(md, sm)[1][:d]) / (2 * e)
        E[t] = np.abs(H) @ (unit * ref["sb"][t, w, :d]) + 16 * unit * G[t]
    Jn = ref["Jn"][:, sl, :d]
    return np.einsum("tak,tk->ta", Jn, E), np.einsum("tak,tk->ta", Jn, G)


def check_moves(specs, md, streams, frames, X, ref, unit=P.U32, tol_f=P.TOL_F, keep=None):
    """The GPU's move of every step and atom against the oracle's next
    frame: the rounding of the position (both sides), the step's force error
    (the per-step force allowance of tests/parity.py for the bias, the
    potential's own floor) times dt mu, and the noise's rounding."""
    c1 = md["dt"] * md["mu"]
    c2 = math.sqrt(2 * md["mu"] * md["kT"] * md["dt"])
    off = synth.offsets_of(specs)
    T = X.shape[0]
    worst = 0.0
    for w, sp in enumerate(specs):
        d = len(sp["grid"]["n"])
        sl = slice(off[w], off[w] + sp["natoms"])
        xi = np.array([[oracle.md_normals(md["seed"], streams[w], t, i) for i in range(sp["natoms"])]
                       for t in range(T)])
        fU_floor, fU = _potential_floor(md, ref, sl, w, d, unit)
        Fb = np.linalg.norm(ref["F"][:, sl], axis=-1)
        scale = (Fb + fU).max(axis=-1, keepdims=True)
        allowF = tol_f * scale + P.force_floor(ref, w, sl, d, unit) + fU_floor + 8 * unit * (Fb + fU)
        xn = frames[1:T + 1, sl]
        allow = (4 * unit * np.linalg.norm(xn, axis=-1) + c1 * allowF
                 + 16 * unit * c2 * np.linalg.norm(xi, axis=-1))
        err = np.linalg.norm(X[:, sl] - xn, axis=-1)
        r = err / allow
        if keep is not None:  # [T, walkers]: steps to check (mABP: not a look-up tie)
            r = np.where(keep[:, w, None], r, 0.0)
        t, i = np.unravel_index(np.argmax(r), r.shape)
        assert r.max() <= 1.0, (w, int(t), int(i), float(err[t, i]), float(allow[t, i]))
        worst = max(worst, float(r.max()))
    return worst


def _oracle_closed_loop(specs, x0, md, streams, T, shared=False):
    ws = [oracle.Walker(s) for s in specs]
    fields = [ws[0].new_field()] * len(ws) if shared else None
    res = oracle.md_run(ws, x0.astype(np.float64), synth.offsets_of(specs), md, streams, 0, T, fields=fields,
                        record_x=True)
    return np.concatenate([res["X"], res["x"][None]])


# ---------------------------------------------------------------- against the oracle, step by step


def test_closed_loop_steps_match_the_oracle_fp32_mueller_brown(abp, ctx):
    """Six COM-distance + dihedral walkers on their own 256 x 256 grids
    under the scaled Mueller-Brown surface (the 64-walker workload's
    dynamics), 150 steps, a deposit every 5 steps."""
    nw, T = 6, 150
    specs = synth.mb64_specs(nw=nw, stride=5)
    md = synth.md_muller_brown(seed=5, state_f32=True)
    streams = np.arange(nw) + 100
    x0 = synth.SweepFrames(nw, seed=21).frames(0, 1)[0]
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    assert np.array_equal(frames.astype(np.float32).astype(np.float64), frames)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    _, ref = oracle_replay(specs, frames[:T].astype(np.float32), 0)
    worst = check_run(abp, ctx, specs, walkers, frames[:T], 0, F, ref)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref)
    print("worst", worst)
    P.record_errors("64 walkers, 2 CVs (closed loop, Mueller-Brown)",
                    "test_closed_loop_steps_match_the_oracle_fp32_mueller_brown", worst)
    # the walkers did move through the potential: the CVs changed
    assert np.ptp(ref["s"][:, :, 0]) > 0.01 and np.ptp(ref["s"][:, :, 1]) > 0.05


@pytest.mark.parametrize("dim", [1, 3])
def test_closed_loop_steps_match_the_oracle_one_and_three_cvs(abp, ctx, dim):
    """The register-fed closed loop with one CV (COM distance, FP32, under
    the double well U = 5 (s^2 - 1)^2) and with three (COM distance,
    dihedral and a second COM distance on a 24^3 grid, under the scaled
    Mueller-Brown surface of the first two), step by step along the
    oracle's trajectory: bias forces, deposits and grids within the
    open-loop tolerances, every move within the error of one FP32 move."""
    nw, T = 4, 120
    if dim == 1:
        specs = [dict(synth.double_well_com_spec(stride=4)) for _ in range(nw)]
        md = synth.md_double_well(seed=6, state_f32=True, mu=0.2)
        x0 = np.concatenate([synth.double_well_com_coords(40 + i) for i in range(nw)]).astype(np.float32)
    else:
        specs = (_equivalence_case(3)[0] + _equivalence_case(3)[0])[:nw]
        md = synth.md_muller_brown(seed=6, state_f32=True)
        x0 = synth.SweepFrames(nw, seed=31).frames(0, 1)[0]
    streams = np.arange(nw) + 200
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    assert np.array_equal(frames.astype(np.float32).astype(np.float64), frames)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    _, ref = oracle_replay(specs, frames[:T].astype(np.float32), 0)
    worst = check_run(abp, ctx, specs, walkers, frames[:T], 0, F, ref)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref)
    print("worst", worst)
    P.record_errors(f"closed loop, {dim} CV{'s' if dim > 1 else ''} (FP32, register-fed form)",
                    f"test_closed_loop_steps_match_the_oracle_one_and_three_cvs[{dim}]", worst)
    assert np.ptp(ref["s"][:, :, 0]) > 0.005


def test_closed_loop_mabp_steps_match_the_oracle(abp, ctx):
    """The paper's own method in the closed loop: mABP with compact S_a^p
    hills (a = 10 grid spacings, p = 20) at the paper's b = 0.9, c = 0.001,
    a hill every second step, on COM-distance + dihedral walkers under the
    scaled Mueller-Brown surface, 150 steps along the oracle's trajectory.
    Deposits (nearest nodes, fixed heights), grids and forces as in the
    open-loop mABP tests (a step whose CV sits in the tie band of a half-node
    may pick the other nearest node, and is left out); every other move
    within the error of one FP32 move."""
    from tests.test_mabp_gpu import _lookup_tie_steps, _mabp, check_mabp

    nw, T = 4, 150
    specs = _mabp(synth.mb64_specs(nw=nw), a_bins=10.0, b=0.9, c=0.001, stride=2)
    md = synth.md_muller_brown(seed=9, state_f32=True)
    streams = np.arange(nw) + 300
    x0 = synth.SweepFrames(nw, seed=41).frames(0, 1)[0]
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    assert np.array_equal(frames.astype(np.float32).astype(np.float64), frames)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    _, ref = oracle_replay(specs, frames[:T].astype(np.float32), 0)
    worst = check_mabp(abp, ctx, specs, walkers, F, ref)
    keep = np.stack([~_lookup_tie_steps(sp, ref["s"][:, i], ref["sb"][:, i]) for i, sp in enumerate(specs)], axis=1)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref, keep=keep)
    print("worst", worst)
    P.record_errors("mABP b = 0.9, c = 0.001, 2 CVs (closed loop, Mueller-Brown)",
                    "test_closed_loop_mabp_steps_match_the_oracle", worst)
    assert np.ptp(ref["s"][:, :, 0]) > 0.005


def test_closed_loop_range_limit_wall_matches_the_oracle(abp, ctx):
    """The CV range limit (a harmonic wall above smax on each CV) in the
    closed loop, register-fed form: walkers that cross the wall on the COM
    distance, step by step along the oracle's trajectory."""
    nw, T = 4, 120
    specs = [dict(sp, hill=synth.with_wall(sp["hill"], [1.5, 3.5], 30.0)) for sp in synth.mb64_specs(nw=nw, stride=4)]
    md = synth.md_muller_brown(seed=10, state_f32=True)
    streams = np.arange(nw) + 400
    x0 = synth.SweepFrames(nw, seed=43).frames(0, 1)[0]
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    _, ref = oracle_replay(specs, frames[:T].astype(np.float32), 0)
    assert np.any(ref["s"][:, :, 0] > 1.5) and np.any(ref["s"][:, :, 0] < 1.5)
    # a walker whose dihedral atoms come close to a line has an FP32 angle
    # whose rounding bound (the oracle's sb) is many times the other walkers':
    # its hills move by more than the fixed grid target allows, so its grid
    # and forces are left to the move check, which carries that bound
    sbmax = ref["sb"].max(axis=0)[:, 1]
    skip = {i for i in range(nw) if sbmax[i] > 10 * np.median(sbmax)}
    assert len(skip) < nw // 2, sbmax
    worst = check_run(abp, ctx, specs, walkers, frames[:T], 0, F, ref, skip=skip)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref)
    print("worst", worst, "ill-conditioned walkers", sorted(skip))


def test_closed_loop_papers_rmsd_setup_matches_the_oracle(abp, ctx):
    """The paper's ligand-run shape in the closed loop (generic form): two
    offset-RMSD CVs of 4 atoms each on the 480 x 480 grid over [0, 12] nm,
    mABP with compact hills a = 10 spacings, p = 20, b = 0.9, c = 0.001, a
    hill every step; free overdamped Langevin of the atoms (no CV
    potential), 150 steps along the oracle's trajectory."""
    from tests.test_mabp_gpu import _lookup_tie_steps, check_mabp

    nw, T = 4, 150
    specs = synth.paper_rmsd_specs(nw=nw)
    md = synth.md_params(seed=12, mu=0.1, state_f32=True)
    streams = np.arange(nw) + 500
    x0 = synth.RmsdFrames(specs, seed=7).frames(0, 1)[0]
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    assert np.array_equal(frames.astype(np.float32).astype(np.float64), frames)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    _, ref = oracle_replay(specs, frames[:T].astype(np.float32), 0)
    worst = check_mabp(abp, ctx, specs, walkers, F, ref)
    keep = np.stack([~_lookup_tie_steps(sp, ref["s"][:, i], ref["sb"][:, i]) for i, sp in enumerate(specs)], axis=1)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref, keep=keep)
    print("worst", worst)
    P.record_errors("paper's RMSD setup, mABP b = 0.9, c = 0.001 (closed loop)",
                    "test_closed_loop_papers_rmsd_setup_matches_the_oracle", worst)
    assert np.ptp(ref["s"][:, :, 0]) > 0.01


def test_closed_loop_full_size_64_walkers(abp, ctx):
    """The benchmark's closed-loop workload at full size: all 64 walkers
    (36 atoms, own 256 x 256 grids, Mueller-Brown x 0.1, mu = 0.1, stride
    50), 120 steps compared with the oracle step by step on the oracle's own
    trajectory; and the benchmark's launch configuration (one launch of many
    steps) gives the same bits as one launch per step for all 64 walkers."""
    nw, T = 64, 120
    specs = synth.mb64_specs(nw=nw)
    md = synth.md_muller_brown(seed=2024, mu=0.1, state_f32=True)
    streams = np.arange(nw)
    x0 = synth.SweepFrames(nw, seed=2031).frames(0, 1)[0]
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    _, ref = oracle_replay(specs, frames[:T].astype(np.float32), 0)
    worst = check_run(abp, ctx, specs, walkers, frames[:T], 0, F, ref)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref)
    print("worst", worst)
    P.record_errors("64 walkers, 2 CVs (closed loop, full size, 64 walkers)", "test_closed_loop_full_size_64_walkers",
                    worst)
    # one launch of T steps against T one-step launches, all 64 walkers
    runs = []
    for chunks in (1, T):
        w = ctx.make_walkers(specs)
        runs.append(gpu_run(abp, ctx, w, x0, md, streams, 0, T, chunks=chunks) + ([ctx.bias(v) for v in w],))
    for a, b in zip(runs[0][:3], runs[1][:3]):
        assert np.array_equal(a, b)
    assert all(np.array_equal(a, b) for a, b in zip(runs[0][3], runs[1][3]))


def test_closed_loop_steps_match_the_oracle_fp64_double_well(abp, ctx):
    """The one-walker FP64 workload (COM distance of two 8-atom groups on
    U = 5 (s^2 - 1)^2, mu = 1), two walkers, 300 steps, a deposit every 10."""
    T = 300
    specs = [synth.double_well_com_spec(stride=10), synth.double_well_com_spec(stride=10)]
    md = synth.md_double_well(seed=9)
    streams = [3, 4]
    x0 = np.concatenate([synth.double_well_com_coords(21), synth.double_well_com_coords(22)])
    frames = _oracle_closed_loop(specs, x0, md, streams, T)
    walkers = ctx.make_walkers(specs, precision=abp.ABP_PREC_FP64)
    abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams, dtype=np.float64)
    _, ref = oracle_replay(specs, frames[:T], 0)
    log = abp.abp_deposit_log_readout(ctx.handle, 1 << 16)
    ids = {w.id: i for i, w in enumerate(walkers)}
    assert not P.compare_deposits(specs, log, ref["deposits"], ids, sb=ref["sb"], unit=P.U64)
    worst = {"V": 0.0, "dV": 0.0, "F": 0.0, "F_step": 0.0, "F_allow": 0.0, "floor_steps": 0}
    for i, w in enumerate(walkers):
        e = P.rel_field_err(ctx.bias(w), ref["fields"][i])
        assert np.all(e < 1e-10)
        sl = slice(16 * i, 16 * i + 16)
        rel, ratio, nfloor = P.check_forces_per_step(F, ref, i, sl, 1, tol=1e-9, unit=P.U64)
        worst["V"] = max(worst["V"], e[0])
        worst["dV"] = max(worst["dV"], e[1:].max())
        worst["F"] = max(worst["F"], P.force_err(F[:, sl], ref["F"][:, sl]))
        worst["F_step"] = max(worst["F_step"], rel)
        worst["F_allow"] = max(worst["F_allow"], ratio)
        worst["floor_steps"] += nfloor
    worst["move"] = check_moves(specs, md, streams, frames, X, ref, unit=P.U64, tol_f=1e-9)
    print("worst", worst)
    P.record_errors("1 walker FP64, double well (closed loop)",
                    "test_closed_loop_steps_match_the_oracle_fp64_double_well", worst)


def test_closed_loop_phased_form_on_a_shared_grid(abp, ctx):
    """Four walkers of the shared-grid workload's shape (COM distance,
    dihedral, CN over 20 x 300 atoms in a 3 nm periodic box) depositing into
    one 40^3 grid, free overdamped Langevin (no CV potential), 12 steps."""
    nw, T = 4, 12
    specs = synth.shared256_specs(nw=nw, n=40, n_lig=20, n_env=300, box=3.0, stride=2, cn_range=(60.0, 160.0))
    md = synth.md_params(seed=13, mu=0.05, state_f32=True)
    streams = np.arange(nw)
    x0 = np.concatenate(synth.shared256_templates(9, nw=nw, n_lig=20, n_env=300, box=3.0)).astype(np.float32)
    frames = _oracle_closed_loop(specs, x0, md, streams, T, shared=True)
    walkers = ctx.make_walkers(specs)
    abp.abp_deposit_log_enable(ctx.handle, 4096)
    X, F = gpu_steps_from(abp, ctx, walkers, frames[:T], md, streams)
    ws = [oracle.Walker(s) for s in specs]
    shared = ws[0].new_field()
    ref = oracle.run(ws, frames[:T], synth.offsets_of(specs), 0, T, fields=[shared] * nw, error_model=True)
    worst = check_run(abp, ctx, specs, walkers, frames[:T], 0, F, ref)
    worst["move"] = check_moves(specs, md, streams, frames, X, ref)
    print("worst", worst)
    P.record_errors("shared grid, phased form (closed loop, 4 walkers on 40^3)",
                    "test_closed_loop_phased_form_on_a_shared_grid", worst)


# ---------------------------------------------------------------- the GPU's own closed loop


def test_launch_length_does_not_change_the_bits(abp, ctx):
    """One launch of 120 steps, four launches, and 120 one-step calls give
    the same trajectory, forces and grids bit for bit."""
    nw, T = 5, 120
    specs = synth.mb64_specs(nw=nw, stride=7)
    md = synth.md_muller_brown(seed=17)
    streams = np.arange(nw) * 7
    x0 = synth.SweepFrames(nw, seed=23).frames(0, 1)[0]
    runs = []
    for chunks in (1, 4, T):
        w = ctx.make_walkers(specs)
        tr, F, xf = gpu_run(abp, ctx, w, x0, md, streams, 0, T, chunks=chunks)
        runs.append((tr, F, xf, [ctx.bias(x) for x in w]))
    for tr, F, xf, B in runs[1:]:
        assert np.array_equal(tr, runs[0][0]) and np.array_equal(F, runs[0][1]) and np.array_equal(xf, runs[0][2])
        for a, b in zip(B, runs[0][3]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("shared", [False, True])
def test_closed_loop_under_cuda_graph_capture(abp, ctx, shared):
    """abp_md_run captured in a CUDA graph (after a direct call has cached
    the walker table) replays the same steps as direct calls: bit for bit in
    the fused closed loop on own grids, to FP64 rounding in the phased form
    on a shared grid (six launches per step; FP64 atomics add a step's hills
    in any order)."""
    if shared:
        nw = 3
        specs = synth.shared256_specs(nw=nw, n=32, n_lig=16, n_env=200, box=3.0, stride=2, cn_range=(30.0, 130.0))
        x0 = np.concatenate(synth.shared256_templates(11, nw=nw, n_lig=16, n_env=200, box=3.0)).astype(np.float32)
        md = synth.md_params(seed=7, mu=0.05)
    else:
        nw = 4
        specs = synth.mb64_specs(nw=nw, stride=3)
        x0 = synth.SweepFrames(nw, seed=29).frames(0, 1)[0]
        md = synth.md_muller_brown(seed=7)
    streams = np.arange(nw) + 5
    T = 12
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    # direct calls: step 0, then steps 1 .. T-1
    wd = ctx.make_walkers(specs)
    xd = abp.to_records(x0[None]).cuda()[0]
    abp.abp_md_run(ctx.handle, wd, xd, abp.ABP_F32, offs, md, streams, step0=0, nsteps=1)
    abp.abp_md_run(ctx.handle, wd, xd, abp.ABP_F32, offs, md, streams, step0=1, nsteps=T - 1)
    torch.cuda.synchronize()
    # step 0 directly (caches the table), steps 1 .. T-1 from a captured graph
    if shared:
        for sp in specs:
            sp["shared"] = "graph"
    wg = ctx.make_walkers(specs)
    xg = abp.to_records(x0[None]).cuda()[0]
    abp.abp_md_run(ctx.handle, wg, xg, abp.ABP_F32, offs, md, streams, step0=0, nsteps=1)
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    ctx.set_stream(st.cuda_stream)
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            abp.abp_md_run(ctx.handle, wg, xg, abp.ABP_F32, offs, md, streams, step0=1, nsteps=T - 1)
        g.replay()
        torch.cuda.synchronize()
    finally:
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
    assert not torch.equal(xd, abp.to_records(x0[None]).cuda()[0])
    if shared:
        assert torch.allclose(xd, xg, rtol=0, atol=1e-6)
        assert np.all(P.rel_field_err(ctx.bias(wg[0]), ctx.bias(wd[0])) < 1e-9)
    else:
        assert torch.equal(xd, xg)
        for a, b in zip(wd, wg):
            assert np.array_equal(ctx.bias(a), ctx.bias(b))


def test_open_loop_replay_of_the_closed_loop_trajectory(abp, ctx):
    """The windowed form (abp_run) replayed on the GPU's own closed-loop
    trajectory computes the closed loop's bias forces and grids: the two
    forms run a step through the same operations."""
    nw, T = 6, 300
    specs = synth.mb64_specs(nw=nw, stride=10)
    md = synth.md_muller_brown(seed=19)
    streams = np.arange(nw)
    x0 = synth.SweepFrames(nw, seed=25).frames(0, 1)[0]
    wm = ctx.make_walkers(specs)
    traj, F, _ = gpu_run(abp, ctx, wm, x0, md, streams, 0, T, chunks=2)
    ww = ctx.make_walkers(specs)
    Fw = gpu_replay(abp, ctx, ww, traj.astype(np.float32), 0, chunks=2)
    assert P.force_err(Fw, F) < 1e-6
    for a, b in zip(wm, ww):
        assert np.all(P.rel_field_err(ctx.bias(a), ctx.bias(b)) < 1e-6)
    print("bitwise equal:", np.array_equal(Fw, F), all(np.array_equal(ctx.bias(a), ctx.bias(b)) for a, b in zip(wm, ww)))


def test_well_tempered_limit_of_the_closed_loop_on_the_gpu(abp, ctx):
    """Four FP64 walkers of the one-walker workload closed on the GPU (COM
    distance of two 8-atom groups, U = 5 (s^2 - 1)^2, mu = 1, kT = 2.5,
    gamma = 10, stride 100), 2e5 steps each: every walker's bias matches
    -(1 - 1/gamma) (U(s) - 2 kT ln s) + C within 0.5 kT RMS on [0.3, 1.7]
    (the free energy of the distance of two freely diffusing centres)."""
    kT, gamma, nw, T = 2.5, 10.0, 4, 200_000
    specs = [synth.double_well_com_spec() for _ in range(nw)]
    md = synth.md_double_well(seed=31)
    x0 = np.concatenate([synth.double_well_com_coords(40 + i) for i in range(nw)])
    walkers = ctx.make_walkers(specs, precision=abp.ABP_PREC_FP64)
    rec = abp.to_records(x0[None], torch.float64).cuda()[0]
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    for c in range(10):
        abp.abp_md_run(ctx.handle, walkers, rec, abp.ABP_F64, offs, md, np.arange(nw), step0=c * T // 10,
                       nsteps=T // 10)
    abp.abp_sync(ctx.handle)
    xi = np.linspace(-2.0, 2.0, 512)
    sel = (xi > 0.3) & (xi < 1.7)
    Fs = 5.0 * (xi[sel] ** 2 - 1.0) ** 2 - 2.0 * kT * np.log(xi[sel])
    for w in walkers:
        resid = ctx.bias(w)[sel, 0] + (1 - 1 / gamma) * Fs
        rms = np.sqrt(np.mean((resid - resid.mean()) ** 2))
        print("rms / kT", rms / kT)
        assert rms < 0.5 * kT, rms
        st = ctx.readout(w)
        assert st["flags"] & abp.WFLAG_NONFINITE == 0


# ---------------------------------------------------------------- edge cases


def test_closed_loop_rejections_and_non_finite_coordinates(abp, ctx):
    md = synth.md_muller_brown()
    cn = synth.uneven1000_specs(seed=3, nw=1, sizes_2d=(48,), n1d=200, n3d=20)
    w = ctx.make_walkers(cn)
    rec = torch.zeros(cn[0]["natoms"], 4, device="cuda")
    offs = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(abp.AbpError) as e:  # a CN walker of the fused form
        abp.abp_md_run(ctx.handle, w, rec, abp.ABP_F32, offs, md, [0])
    assert e.value.code == abp.ABP_ERR_UNSUPPORTED
    one = ctx.make_walkers([synth.double_well_com_spec()])
    with pytest.raises(abp.AbpError) as e:  # Mueller-Brown needs two CVs
        abp.abp_md_run(ctx.handle, one, torch.zeros(16, 4, device="cuda"), abp.ABP_F32, offs, md, [0])
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    with pytest.raises(abp.AbpError) as e:
        abp.abp_md_run(ctx.handle, one, torch.zeros(16, 4, device="cuda"), abp.ABP_F32, offs,
                       synth.md_params(dt=-1.0), [0])
    assert e.value.code == abp.ABP_ERR_INVALID_ARG
    shared = synth.shared256_specs(nw=2, n=24, n_lig=8, n_env=40, box=3.0, stride=2, cn_range=(0.0, 40.0))
    sw = ctx.make_walkers(shared)
    offs2 = torch.tensor(synth.offsets_of(shared), dtype=torch.int64, device="cuda")
    with pytest.raises(abp.AbpError) as e:  # the phased form takes no CV potential
        abp.abp_md_run(ctx.handle, sw, torch.zeros(96, 4, device="cuda"), abp.ABP_F32, offs2,
                       synth.md_double_well(), [0, 1])
    assert e.value.code == abp.ABP_ERR_UNSUPPORTED
    # non-finite coordinates: that walker stops (its atoms stay as they were),
    # the other runs on
    specs = synth.mb64_specs(nw=2, stride=3)
    walkers = ctx.make_walkers(specs)
    x0 = synth.SweepFrames(2, seed=2).frames(0, 1)[0].copy()
    x0[5, 1] = np.nan
    buf = abp.to_records(x0[None]).cuda()[0]
    before = buf.clone()
    offs3 = torch.tensor([0, 36], dtype=torch.int64, device="cuda")
    abp.abp_md_run(ctx.handle, walkers, buf, abp.ABP_F32, offs3, md, [0, 1], nsteps=5)
    with pytest.raises(abp.AbpError) as e:
        abp.abp_sync(ctx.handle)
    assert e.value.code == abp.ABP_ERR_NONFINITE
    assert torch.equal(torch.nan_to_num(buf[:36]), torch.nan_to_num(before[:36]))
    assert not torch.equal(buf[36:], before[36:])
    assert ctx.readout(walkers[0])["flags"] == abp.WFLAG_NONFINITE
    assert np.all(ctx.bias(walkers[0]) == 0.0)


@pytest.mark.gpu
def test_closed_loop_walker_that_blows_up_mid_launch_reports_it(abp, ctx):
    """A walker whose coordinates overflow after some completed steps stops
    at the first non-finite ones: the call reports it and the walker's state
    says ABP_WFLAG_NONFINITE (its values are its last completed step's). The
    double well's force, scaled by 1e30 on the first CV, takes the atoms past
    the FP32 range within a few steps."""
    specs = synth.mb64_specs(nw=2, stride=3)
    walkers = ctx.make_walkers(specs)
    x0 = synth.SweepFrames(2, seed=2).frames(0, 1)[0]
    buf = abp.to_records(x0[None]).cuda()[0]
    offs = torch.tensor([0, 36], dtype=torch.int64, device="cuda")
    md = synth.md_double_well(seed=4, A=1e30, B=0.1)
    abp.abp_md_run(ctx.handle, walkers, buf, abp.ABP_F32, offs, md, [0, 1], nsteps=20)
    with pytest.raises(abp.AbpError) as e:
        abp.abp_sync(ctx.handle)
    assert e.value.code == abp.ABP_ERR_NONFINITE
    x = buf.cpu().numpy()[:, :3]
    for i, w in enumerate(walkers):
        r = ctx.readout(w)
        assert r["flags"] == abp.WFLAG_NONFINITE, r
        assert not np.all(np.isfinite(x[36 * i:36 * (i + 1)]))
        # the first step deposited before the blow-up
        assert np.any(ctx.bias(w)[:, 0] != 0.0)


def test_closed_loop_checkpoint_and_resume_is_bit_exact(abp, ctx):
    """The closed loop's state is the grid, the coordinates and the step
    counter (the deposit schedule and the Philox counters follow from the
    step): save the grids after k closed-loop steps (abp_grid_save), restore
    them into new walkers and continue from the saved coordinates at step k;
    the coordinates, the bias forces and the grids equal an uninterrupted run
    bit for bit. Two walker sets: the register-fed form (COM groups of 16,
    a dihedral) and the generic one (an RMSD CV)."""
    rmsd = []
    for sp in synth.mb64_specs(nw=2, stride=3):
        sp = dict(sp)
        ref = synth.SweepFrames(1, seed=21).frames(0, 1)[0][32:36].astype(np.float64)
        sp["cvs"] = [sp["cvs"][0], {"type": "rmsd", "a": np.arange(32, 36), "ref": ref}]
        sp["grid"] = synth.grid((0.2, 0.0), (2.0, 1.0), (256, 256), (False, False))
        sp["hill"] = synth.hill(0.5, (0.04, 0.04), 3, 15.0)
        rmsd.append(sp)
    md = synth.md_muller_brown(seed=6, mu=0.1)
    for specs in (synth.mb64_specs(nw=2, stride=3), rmsd):
        x0 = abp.to_records(synth.SweepFrames(2, seed=17).frames(0, 1)[0][None]).cuda()[0]
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        n, k = 40, 23
        wa = ctx.make_walkers(specs)
        xa = x0.clone()
        Fa = torch.zeros(n, xa.shape[0], 4, device="cuda")
        abp.abp_md_run(ctx.handle, wa, xa, abp.ABP_F32, offs, md, [0, 1], forces=Fa, force_offsets=offs,
                       force_step_stride=xa.shape[0], step0=0, nsteps=n)
        wb = ctx.make_walkers(specs)
        xb = x0.clone()
        abp.abp_md_run(ctx.handle, wb, xb, abp.ABP_F32, offs, md, [0, 1], step0=0, nsteps=k)
        torch.cuda.synchronize()
        saved = [abp.abp_grid_save(ctx.handle, w.grid) for w in wb]
        wc = ctx.make_walkers(specs)
        for w, g in zip(wc, saved):
            abp.abp_grid_restore(ctx.handle, w.grid, g)
        Fc = torch.zeros(n - k, xb.shape[0], 4, device="cuda")
        abp.abp_md_run(ctx.handle, wc, xb, abp.ABP_F32, offs, md, [0, 1], forces=Fc, force_offsets=offs,
                       force_step_stride=xb.shape[0], step0=k, nsteps=n - k)
        torch.cuda.synchronize()
        assert torch.equal(xa, xb)
        assert torch.equal(Fa[k:], Fc)
        for x, y in zip(wa, wc):
            assert np.array_equal(ctx.bias(x), ctx.bias(y))


def _rmsd_spec(seed=21):
    """A two-CV walker (COM distance + a 4-atom RMSD) that the closed loop
    runs in its generic form."""
    sp = dict(synth.mb64_specs(nw=1, stride=3)[0])
    ref = synth.SweepFrames(1, seed=seed).frames(0, 1)[0][32:36].astype(np.float64)
    sp["cvs"] = [sp["cvs"][0], {"type": "rmsd", "a": np.arange(32, 36), "ref": ref}]
    sp["grid"] = synth.grid((0.2, 0.0), (2.0, 1.0), (256, 256), (False, False))
    sp["hill"] = synth.hill(0.5, (0.04, 0.04), 3, 15.0)
    return sp


def _equivalence_case(dim):
    """Walkers of the register-fed form for `dim` CVs, a walker of the same
    dimension that is not (an RMSD CV), the dynamics, and the atoms per
    walker."""
    if dim == 1:
        fast = [dict(synth.double_well_com_spec(stride=3)) for _ in range(3)]
        ref = synth.SweepFrames(1, seed=22).frames(0, 1)[0][:4].astype(np.float64)
        other = {"natoms": 16, "cvs": [{"type": "rmsd", "a": np.arange(0, 4), "ref": ref}],
                 "grid": synth.grid((0.0,), (2.0,), (512,), (False,)), "hill": synth.hill(0.5, (0.05,), 3, 10.0)}
        return fast, other, synth.md_params(seed=8, mu=0.1), 16
    if dim == 2:
        return synth.mb64_specs(nw=3, stride=3), _rmsd_spec(), synth.md_muller_brown(seed=8, mu=0.1), 36
    g3 = synth.grid((0.2, -math.pi, 0.0), (2.0, math.pi, 1.5), (24, 24, 24), (False, True, False))
    h3 = synth.hill(0.5, (0.1, 0.3, 0.1), 3, 15.0)
    base = synth.mb64_specs(nw=1)[0]
    fast = []
    for _ in range(3):
        sp = dict(base)
        sp["cvs"] = list(base["cvs"]) + [{"type": "com_dist", "a": np.arange(0, 8), "b": np.arange(8, 16)}]
        sp["grid"], sp["hill"] = g3, h3
        fast.append(sp)
    ref = synth.SweepFrames(1, seed=23).frames(0, 1)[0][16:20].astype(np.float64)
    other = dict(base)
    other["cvs"] = list(base["cvs"]) + [{"type": "rmsd", "a": np.arange(16, 20), "ref": ref}]
    other["grid"], other["hill"] = g3, h3
    return fast, other, synth.md_muller_brown(seed=8, mu=0.1), 36


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_register_fed_form_gives_the_generic_forms_bits(abp, ctx, dim):
    """The register-fed instantiation of the closed-loop kernel (chosen when
    every walker of a launch qualifies) computes the same operations as the
    generic one: the same COM-distance / dihedral walkers run alone (the
    register-fed form) and beside an RMSD walker of the same dimension (which
    sends the whole launch to the generic form) give the same coordinates,
    bias forces, grids and walker states bit for bit, over 60 steps with
    deposits every third step; one, two and three CVs."""
    specs, other, md, na = _equivalence_case(dim)
    n = 60
    x0 = synth.SweepFrames(4, seed=19).frames(0, 1)[0].reshape(4, 36, 3)[:, :na].reshape(-1, 3)
    nf = 3 * na
    wf = ctx.make_walkers(specs)
    xf = abp.to_records(x0[None, :nf]).cuda()[0]
    of = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    Ff = torch.zeros(n, nf, 4, device="cuda")
    abp.abp_md_run(ctx.handle, wf, xf, abp.ABP_F32, of, md, [0, 1, 2], forces=Ff, force_offsets=of,
                   force_step_stride=nf, step0=0, nsteps=n)
    mixed = list(specs) + [other]
    wg = ctx.make_walkers(mixed)
    xg = abp.to_records(x0[None]).cuda()[0]
    og = torch.tensor(synth.offsets_of(mixed), dtype=torch.int64, device="cuda")
    Fg = torch.zeros(n, xg.shape[0], 4, device="cuda")
    abp.abp_md_run(ctx.handle, wg, xg, abp.ABP_F32, og, md, [0, 1, 2, 3], forces=Fg, force_offsets=og,
                   force_step_stride=xg.shape[0], step0=0, nsteps=n)
    torch.cuda.synchronize()
    assert not torch.equal(xf, abp.to_records(x0[None, :nf]).cuda()[0])
    assert torch.equal(xf, xg[:nf])
    assert torch.equal(Ff, Fg[:, :nf])
    for a, b in zip(wf, wg[:3]):
        assert np.array_equal(ctx.bias(a), ctx.bias(b))
        ra, rb = ctx.readout(a), ctx.readout(b)
        for key in ("s", "V", "dV", "flags"):
            assert np.array_equal(np.asarray(ra[key]), np.asarray(rb[key])), key
