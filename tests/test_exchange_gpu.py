"""GPU hill exchange for walkers that share one bias across devices
(abp_shared_hills, abp_grid_apply_hills, abp_shared_forces), on one GPU.

Two replicas of the shared grid hold three and two walkers of a five-walker
run and swap their hill records on the host, as two ranks do through
``exchange.gather_hills``; a third grid runs all five walkers. The replicas
must stay bit-identical to each other and to the single grid (records are
applied in list order, no atomics), and the single grid must match the FP64
oracle run of the five walkers on one shared grid. A batch of records
applied in one call must equal the same records applied one call each."""
import math

import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import exchange, synth
from tests import parity as P
from tests.test_parity_gpu import check_run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT = (0, 3, 5)
T = 7


@pytest.fixture(scope="module")
def abp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import abp as A
    from paper_1609_09833_gb300 import build

    build.build()
    A.load()
    return A


def _specs(n=40, key="shared256"):
    specs = synth.shared256_specs(nw=SPLIT[-1], n=n, n_lig=20, n_env=300, box=3.0, stride=2,
                                  cn_range=(60.0, 160.0))
    out = []
    for i, sp in enumerate(specs):
        sp = dict(sp, shared=key)
        if i >= SPLIT[1]:
            sp["hill"] = dict(sp["hill"], stride=3)
        out.append(sp)
    return out


def test_two_replicas_equal_one_shared_grid(abp):
    specs = _specs()
    tm = synth.shared256_templates(9, nw=len(specs), n_lig=20, n_env=300, box=3.0)
    frames = synth.JitterFrames(tm, seed=10, jitter=0.01).frames(0, T)
    ctx, ctx_r = abp.Context(0), abp.Context(0)
    try:
        wa = ctx.make_walkers([dict(s, shared="replica0") for s in specs[: SPLIT[1]]])
        wb = ctx.make_walkers([dict(s, shared="replica1") for s in specs[SPLIT[1]:]])
        abp.abp_deposit_log_enable(ctx_r.handle, 4096)
        wr = ctx_r.make_walkers(specs)
        ra, rb, rr = exchange.GpuReplica(ctx, wa), exchange.GpuReplica(ctx, wb), exchange.GpuReplica(ctx_r, wr)
        rec = abp.to_records(frames).cuda()
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        oa, ob = offs[: SPLIT[1]], offs[SPLIT[1]:]
        Fab, Fr = torch.zeros_like(rec), torch.zeros_like(rec)
        counts = []
        for t in range(T):
            every = np.concatenate([ra.hills(rec[t], oa, t), rb.hills(rec[t], ob, t)])
            hr = exchange.shared_step(rr, rec[t], offs, Fr[t], offs, t)  # one rank: the local records
            for key in ("s", "height", "step"):
                assert np.array_equal(every[key], hr[key]), (t, key)
            if len(every):
                ra.apply(every)
                rb.apply(every)
            ra.forces(Fab[t], oa, abp.ABP_FORCES_OVERWRITE, t)
            rb.forces(Fab[t], ob, abp.ABP_FORCES_OVERWRITE, t)
            counts.append(len(every))
        torch.cuda.synchronize()
        assert counts == [5, 0, 3, 2, 3, 0, 5]
        assert torch.equal(Fab, Fr)
        ga, gb, gr = ctx.bias(wa[0]), ctx.bias(wb[0]), ctx_r.bias(wr[0])
        assert np.array_equal(ga, gb) and np.array_equal(ga, gr)
        # the single grid against the oracle run of all five walkers
        ws = [oracle.Walker(s) for s in specs]
        shared = ws[0].new_field()
        ref = oracle.run(ws, frames.astype(np.float64), synth.offsets_of(specs), 0, T, fields=[shared] * len(ws),
                         error_model=True)
        Fg = Fr.cpu().numpy()[..., :3].astype(np.float64)
        worst = check_run(abp, ctx_r, specs, wr, frames, 0, Fg, ref)
        print("worst errors", worst)
    finally:
        torch.cuda.synchronize()
        ctx.close()
        ctx_r.close()


def _records(spec, n, seed):
    """Hill records over the grid's range: some beyond the non-periodic
    edges, some at the periodic seam, some on top of one another."""
    g = spec["grid"]
    r = np.random.default_rng(seed)
    h = np.zeros(n, dtype=exchange.HILL_DTYPE)
    lo, hi = np.asarray(g["lo"]), np.asarray(g["hi"])
    span = hi - lo
    s = lo + r.uniform(-0.08, 1.08, size=(n, 3)) * span
    s[: n // 5, 1] = r.choice([-math.pi + 1e-3, math.pi - 1e-3], size=n // 5)  # the seam of the dihedral axis
    if n >= n // 5 + 6:
        s[n // 5: n // 5 + 6] = s[n // 5]  # six hills on one centre
    h["s"] = s
    h["height"] = r.uniform(0.05, 0.3, size=n)
    h["step"] = np.arange(n)
    return h


def test_batched_apply_equals_one_record_at_a_time(abp):
    spec = _specs(n=64)[0]
    recs = _records(spec, 80, seed=3)
    ctx = abp.Context(0)
    try:
        w1 = ctx.make_walkers([dict(spec, shared="batched")])[0]
        w2 = ctx.make_walkers([dict(spec, shared="one_by_one")])[0]
        abp.abp_grid_apply_hills(ctx.handle, w1, recs)
        for i in range(len(recs)):
            abp.abp_grid_apply_hills(ctx.handle, w2, recs[i: i + 1])
        g1, g2 = ctx.bias(w1), ctx.bias(w2)
        assert np.array_equal(g1, g2)
        wo = oracle.Walker(spec)
        f = wo.new_field()
        for r in recs:
            oracle.deposit(wo, f, r["s"], float(r["height"]))
        assert np.all(P.rel_field_err(g1, f) < P.TOL_V)
        assert np.count_nonzero(g1[:, 0]) > 0
    finally:
        torch.cuda.synchronize()
        ctx.close()


def test_exchange_rejects_bad_input(abp):
    spec = _specs(n=32)[0]
    ctx = abp.Context(0)
    try:
        w = ctx.make_walkers([spec])[0]
        own = dict(spec)
        own.pop("shared")
        wo = ctx.make_walkers([own])[0]
        bad = _records(spec, 2, seed=1)
        bad["height"][1] = float("nan")
        with pytest.raises(abp.AbpError) as e:
            abp.abp_grid_apply_hills(ctx.handle, w, bad)
        assert e.value.code == abp.ABP_ERR_INVALID_ARG
        bad = _records(spec, 2, seed=1)
        bad["s"][0, 2] = float("inf")
        with pytest.raises(abp.AbpError):
            abp.abp_grid_apply_hills(ctx.handle, w, bad)
        with pytest.raises(abp.AbpError):  # an unshared grid has no FP64 shadow to apply records to
            abp.abp_grid_apply_hills(ctx.handle, wo, _records(spec, 2, seed=1))
        x = torch.zeros(1, spec["natoms"], 4, device="cuda")
        offs = torch.zeros(1, dtype=torch.int64, device="cuda")
        with pytest.raises(abp.AbpError):
            abp.abp_shared_hills(ctx.handle, [wo], x[0], abp.ABP_F32, offs, 0)
        abp.abp_grid_apply_hills(ctx.handle, w, _records(spec, 0, seed=1))  # nothing to do
        assert np.count_nonzero(ctx.bias(w)) == 0
    finally:
        torch.cuda.synchronize()
        ctx.close()
