"""The serving loop (abp_server_*): continuous batching of single-step
requests from many simulations. Each simulation's result is the same alone
and in any mix (bit for bit: a walker's reductions have a fixed order) and
matches the FP64 oracle; requests of one simulation complete in order;
admission follows the context's HBM budget and resumes as memory frees."""
import time

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


def _frames(tmpl, seed, T):
    r = synth.rng(seed)
    return np.stack([tmpl + r.normal(scale=0.02, size=tmpl.shape) for _ in range(T)]).astype(np.float32)


def _records(x):
    rec = np.zeros(x.shape[:-1] + (4,), dtype=np.float32)
    rec[..., :3] = x
    return np.ascontiguousarray(rec)


def _serve(abp, srv, sims, coords, steps, order):
    """Submit requests in `order` ((sim index, step) pairs) and wait for all."""
    out = {}
    for i, t in order:
        f = np.zeros_like(coords[i][t])
        out[(i, t)] = f
        abp.abp_server_submit(srv, sims[i], steps[t], coords[i][t], f, tag=i * 1000 + t)
    got, deadline = [], time.time() + 60
    while len(got) < len(order) and time.time() < deadline:
        got += abp.abp_server_poll(srv, 4096, wait_ms=50)
    assert len(got) == len(order)
    assert all(r.status == 0 for r in got)
    return out, got


def test_results_alone_and_in_the_mix(abp):
    ctx = abp.Context(0)
    srv = abp.abp_server_create(ctx.handle, max_batch=256, max_atoms=256, nstreams=2)
    try:
        specs = synth.serve_specs(seed=3, nsim=40, side=(64, 160), stride=(2, 5))
        tmpl = synth.serve_templates(3, specs)
        T = 12
        coords = [_records(_frames(t, 100 + i, T)) for i, t in enumerate(tmpl)]
        steps = list(range(T))
        keep = []

        def admit(sp):
            desc, k = abp.walker_desc(sp)
            keep.append(k)
            return abp.abp_server_admit(srv, abp.grid_desc(sp["grid"]), desc)

        # simulation 0 alone (its twin is admitted separately for the mix)
        alone = [admit(specs[0])]
        out_alone, _ = _serve(abp, srv, alone, coords[:1], steps, [(0, t) for t in range(T)])
        mix = [admit(sp) for sp in specs]
        order = [(i, t) for t in range(T) for i in np.random.default_rng(7).permutation(len(specs))]
        out_mix, got = _serve(abp, srv, mix, coords, steps, order)
        for t in range(T):
            assert np.array_equal(out_alone[(0, t)], out_mix[(0, t)])
        # the mix really was batched, and each simulation's steps came back in order
        assert max(r.batch for r in got) > 1
        for i in range(len(specs)):
            seq = [r.step for r in got if r.sim == mix[i]]
            assert seq == sorted(seq)
        # against the oracle, for a few simulations
        for i in (0, 7, 21):
            wo = oracle.Walker(specs[i])
            ref = oracle.run([wo], coords[i][:, :, :3].astype(np.float64), [0], 0, T)
            Fg = np.stack([out_mix[(i, t)][:, :3] for t in range(T)]).astype(np.float64)
            assert P.force_err(Fg, ref["F"]) < P.TOL_F
        st = abp.abp_server_stats(srv)
        assert st["finished"] == st["submitted"] == T * (len(specs) + 1)
        assert st["launches"] < st["finished"]
    finally:
        abp.abp_server_destroy(srv)
        ctx.close()


def test_backlog_pipelines_across_slots_in_order(abp):
    """Several steps of each simulation queued at once (one submit_many call):
    consecutive steps of a simulation run in different launches on different
    streams, ordered on the device, and give the same bits as the same steps
    submitted one at a time, waiting for each result; the results of a
    simulation come back in step order."""
    specs = synth.serve_specs(seed=9, nsim=24, side=(64, 192), stride=(2, 4))
    tmpl = synth.serve_templates(9, specs)
    T = 10
    coords = [_records(_frames(t, 300 + i, T)) for i, t in enumerate(tmpl)]
    outs = []
    for nstreams, backlog in ((2, False), (4, True)):
        ctx = abp.Context(0)
        srv = abp.abp_server_create(ctx.handle, max_batch=64, max_atoms=256, nstreams=nstreams)
        try:
            keep, sims = [], []
            for sp in specs:
                desc, k = abp.walker_desc(sp)
                keep.append(k)
                sims.append(abp.abp_server_admit(srv, abp.grid_desc(sp["grid"]), desc))
            if backlog:
                order = [(i, t) for t in range(T) for i in range(len(specs))]
                packed = np.ascontiguousarray(np.concatenate([coords[i][t] for i, t in order]))
                out = np.zeros_like(packed)
                abp.abp_server_submit_many(srv, [sims[i] for i, _ in order], [t for _, t in order], packed, out)
                got, deadline = [], time.time() + 60
                while len(got) < len(order) and time.time() < deadline:
                    got += abp.abp_server_poll(srv, 4096, wait_ms=50)
                assert len(got) == len(order) and all(r.status == 0 for r in got)
                for i in range(len(specs)):
                    seq = [r.step for r in got if r.sim == sims[i]]
                    assert seq == list(range(T))
                res, off = {}, 0
                for i, t in order:
                    n = coords[i].shape[1]
                    res[(i, t)] = out[off:off + n]
                    off += n
                st = abp.abp_server_stats(srv)
                # fewer launches than steps x simulations: the backlog was batched
                assert st["launches"] < T * len(specs) / 4
            else:
                res = {}
                for t in range(T):  # one step of every simulation, then wait
                    o, _ = _serve(abp, srv, sims, coords, list(range(T)), [(i, t) for i in range(len(specs))])
                    res.update(o)
            outs.append(res)
        finally:
            abp.abp_server_destroy(srv)
            ctx.close()
    assert any(np.any(v != 0) for v in outs[0].values())
    for key in outs[0]:
        assert np.array_equal(outs[0][key], outs[1][key]), key


def test_cancel_drops_the_queued_requests_of_a_simulation(abp):
    """50 steps of one simulation queued at once, then cancelled: the steps
    already launched finish (a prefix, in order, status 0), the rest come back
    cancelled with their force buffers untouched, and the simulation is
    served again afterwards."""
    ctx = abp.Context(0)
    srv = abp.abp_server_create(ctx.handle, max_batch=64, max_atoms=256, nstreams=2)
    try:
        spec = synth.serve_specs(seed=13, nsim=1, side=(256, 256), atoms=(64, 64), stride=(5, 5))[0]
        desc, keep = abp.walker_desc(spec)
        sim = abp.abp_server_admit(srv, abp.grid_desc(spec["grid"]), desc)
        T = 50
        coords = _records(_frames(synth.serve_templates(13, [spec])[0], 5, T + 1))
        packed = np.ascontiguousarray(coords[:T].reshape(-1, 4))
        out = np.full_like(packed, 7.0)
        abp.abp_server_submit_many(srv, [sim] * T, list(range(T)), packed, out)
        n = abp.abp_server_cancel(srv, sim)
        got, deadline = [], time.time() + 60
        while len(got) < T and time.time() < deadline:
            got += abp.abp_server_poll(srv, 4096, wait_ms=50)
        assert len(got) == T
        done = sorted(r.step for r in got if r.status == 0)
        cancelled = sorted(r.step for r in got if r.status == abp.ABP_ERR_CANCELLED)
        assert len(cancelled) == n >= 1
        assert done == list(range(len(done))) and cancelled == list(range(len(done), T))
        F = out.reshape(T, -1, 4)
        assert np.all(F[len(done):] == 7.0)
        assert all(np.any(F[t] != 7.0) for t in range(len(done)))
        f = np.zeros_like(coords[0])
        abp.abp_server_submit(srv, sim, len(done), coords[len(done)], f)
        r = abp.abp_server_poll(srv, 16, wait_ms=5000)
        assert len(r) == 1 and r[0].status == 0 and np.any(f != 0)
        st = abp.abp_server_stats(srv)
        assert st["finished"] == st["submitted"] == T + 1 and st["queued"] == 0
    finally:
        abp.abp_server_destroy(srv)
        ctx.close()


def test_admission_by_hbm_budget(abp):
    ctx = abp.Context(0, budget=40 << 20)
    srv = abp.abp_server_create(ctx.handle, max_batch=64, max_atoms=64, nstreams=2)
    try:
        spec = synth.serve_specs(seed=5, nsim=1, side=(512, 512), atoms=(16, 16))[0]  # 512^2 x 32 B = 8 MB grid
        desc, keep = abp.walker_desc(spec)
        sims = []
        with pytest.raises(abp.AbpError) as e:
            for _ in range(10):
                sims.append(abp.abp_server_admit(srv, abp.grid_desc(spec["grid"]), desc))
        assert e.value.code == abp.ABP_ERR_ADMISSION
        assert 2 <= len(sims) < 10
        x = _records(_frames(synth.serve_templates(5, [spec])[0], 1, 1))[0]
        f = np.zeros_like(x)
        abp.abp_server_submit(srv, sims[0], 0, x, f)
        abp.abp_server_release(srv, sims[0])  # waits for its request, then frees its memory
        sims.append(abp.abp_server_admit(srv, abp.grid_desc(spec["grid"]), desc))
        got = abp.abp_server_poll(srv, 16, wait_ms=1000)
        assert len(got) == 1 and got[0].status == 0
        assert np.any(f != 0)
    finally:
        abp.abp_server_destroy(srv)
        ctx.close()


def test_full_size_simulations_against_the_oracle(abp):
    """The twelve simulations with the largest grids of the served workload
    (sides up to 1024, hills two grid spacings wide, 8 to 256 atoms, its own
    strides), 400 steps each through the server, against the oracle: every
    deposit's CV values, centre and height, every step's forces (with the
    per-step allowance of tests/parity.py) and the grids at the end."""
    from tests.test_parity_gpu import check_run

    specs_all = synth.serve_specs(seed=61, nsim=4096)
    tmpl_all = synth.serve_templates(61, specs_all)
    pick = sorted(range(len(specs_all)), key=lambda i: -specs_all[i]["grid"]["n"][0])[:12]
    specs = [specs_all[i] for i in pick]
    T = 400
    ctx = abp.Context(0)
    srv = abp.abp_server_create(ctx.handle, max_batch=64, max_atoms=256, nstreams=2)
    try:
        abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
        keep, sims = [], []
        for sp in specs:
            desc, k = abp.walker_desc(sp)
            keep.append(k)
            sims.append(abp.abp_server_admit(srv, abp.grid_desc(sp["grid"]), desc))
        coords = [_records(_frames(tmpl_all[i], 500 + i, T)) for i in pick]
        order = [(j, t) for t in range(T) for j in range(len(specs))]
        out, _ = _serve(abp, srv, sims, coords, list(range(T)), order)
        frames = np.concatenate([c[:, :, :3] for c in coords], axis=1).astype(np.float64)
        Fg = np.concatenate([np.stack([out[(j, t)][:, :3] for t in range(T)]) for j in range(len(specs))],
                            axis=1).astype(np.float64)
        ws = [oracle.Walker(sp) for sp in specs]
        ref = oracle.run(ws, frames, synth.offsets_of(specs), 0, T, error_model=True)
        grids = [abp.abp_server_bias_readout(srv, s, sp["grid"]) for s, sp in zip(sims, specs)]

        class _Fields:  # check_run reads each walker's grid through ctx.bias
            def bias(self, w):
                return grids[w.i]

        class _W:
            def __init__(self, i, wid):
                self.id, self.i = wid, i

        log = abp.abp_deposit_log_readout(ctx.handle, 1 << 16)
        ids = sorted(set(int(x) for x in log["walker_id"]))
        assert len(ids) == len(specs)  # every simulation deposited at step 0
        # walker ids in admission order
        walkers = [_W(i, wid) for i, wid in enumerate(ids)]
        worst = check_run(abp, _Fields(), specs, walkers, frames, 0, Fg, ref, log=log)
        print("sides", [sp["grid"]["n"][0] for sp in specs], "worst", worst)
        P.record_errors("serving 4096 simulations (the 12 largest grids, 400 steps through the server)",
                        "test_full_size_simulations_against_the_oracle", worst)
    finally:
        abp.abp_server_destroy(srv)
        ctx.close()
