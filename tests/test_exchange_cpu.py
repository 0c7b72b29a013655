"""Hill exchange across ranks (paper_1609_09833_gb300.exchange) on CPU.

Two gloo ranks hold three and two walkers of one multiple-walker run, each
with its own replica of the shared grid, and step through
``exchange.shared_step`` with a replica backed by the oracle's functions.
After every step the replicas must be bit-identical, and the whole run must
equal, bit for bit, the oracle run of all five walkers on one shared grid
(CVs and heights of a step from the grid before its deposits, deposits in
walker order, forces from the grid after them). The two ranks' walkers
deposit at different strides, so some steps bring hills from one rank only
and some from none."""
import os
import socket
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from paper_1609_09833_gb300 import abp, exchange, synth

SPLIT = (0, 3, 5)
T = 7


class OracleReplica:
    """One rank's walkers and its replica grid, on the oracle's functions.
    ``first`` is the global index of the rank's first walker."""

    def __init__(self, specs, first):
        self.ws = [oracle.Walker(s) for s in specs]
        self.field = self.ws[0].new_field()
        self.first = first

    def hills(self, x, offsets, step):
        self.s, self.J = [], []
        out = []
        for i, w in enumerate(self.ws):
            xi = x[offsets[i]: offsets[i] + w.struct.natoms]
            sv, Jv = zip(*[oracle.cv_eval(w, k, xi)[:2] for k in range(w.d)])
            self.s.append(np.array(sv))
            self.J.append(Jv)
            if step % w.struct.hill.stride == 0:
                Vb = oracle.interp(w, self.field, self.s[-1])[0]
                r = np.zeros(1, dtype=exchange.HILL_DTYPE)
                r["s"][0, : w.d] = self.s[-1]
                r["height"] = oracle.height(w, Vb)
                r["step"] = step
                r["walker_id"] = self.first + i
                out.append(r)
        return np.concatenate(out) if out else np.zeros(0, dtype=exchange.HILL_DTYPE)

    def apply(self, hills):
        w = self.ws[0]
        for r in hills:
            oracle.deposit(w, self.field, r["s"][: w.d], float(r["height"]))

    def forces(self, F, offsets, mode, step):
        for i, w in enumerate(self.ws):
            dV = oracle.interp(w, self.field, self.s[i])[1]
            acc = np.zeros_like(self.J[i][0])
            for k in range(w.d):
                acc = acc + dV[k] * self.J[i][k]
            F[offsets[i]: offsets[i] + w.struct.natoms] = -acc


def _specs():
    specs = synth.shared256_specs(nw=SPLIT[-1], n=28, n_lig=20, n_env=300, box=3.0, stride=2,
                                  cn_range=(60.0, 160.0))
    out = []
    for i, sp in enumerate(specs):
        sp = dict(sp)
        if i >= SPLIT[1]:
            sp["hill"] = dict(sp["hill"], stride=3)
        out.append(sp)
    return out


def _frames(specs):
    tm = synth.shared256_templates(9, nw=len(specs), n_lig=20, n_env=300, box=3.0)
    return synth.JitterFrames(tm, seed=10, jitter=0.01).frames(0, T).astype(np.float64)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        specs = _specs()
        frames = _frames(specs)
        lo, hi = SPLIT[rank], SPLIT[rank + 1]
        offs = np.append(np.asarray(synth.offsets_of(specs), dtype=np.int64), frames.shape[1])
        loc = offs[lo:hi] - offs[lo]
        rep = OracleReplica(specs[lo:hi], lo)
        F, hills, fields = [], [], []
        for t in range(T):
            x = frames[t, offs[lo]: offs[hi]]
            f = np.zeros_like(x)
            hills.append(exchange.shared_step(rep, x, loc, f, loc, t))
            F.append(f)
            fields.append(rep.field.copy())
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), F=np.stack(F), fields=np.stack(fields),
                 hills=np.concatenate(hills), counts=np.array([len(h) for h in hills]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_equal_one_shared_grid(tmp_path):
    pytest.importorskip("torch.distributed")
    oracle.lib()  # build once, before the ranks start
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert [p.exitcode for p in procs] == [0, 0]
    r0, r1 = (np.load(tmp_path / f"rank{r}.npz") for r in range(2))

    # both ranks applied the same records, in the same order, to equal replicas
    assert np.array_equal(r0["hills"].view(np.uint8), r1["hills"].view(np.uint8))
    assert np.array_equal(r0["fields"], r1["fields"])
    # steps with hills from both ranks, from one only, and from none
    assert list(r0["counts"]) == [5, 0, 3, 2, 3, 0, 5]

    specs = _specs()
    frames = _frames(specs)
    ws = [oracle.Walker(s) for s in specs]
    shared = ws[0].new_field()
    ref = oracle.run(ws, frames, synth.offsets_of(specs), 0, T, fields=[shared] * len(ws))
    assert np.array_equal(r0["fields"][-1], shared)
    dep = ref["deposits"]
    h = r0["hills"]
    assert np.array_equal(h["step"], dep["step"])
    assert np.array_equal(h["walker_id"], dep["walker"])
    assert np.array_equal(h["s"], dep["s"])
    assert np.array_equal(h["height"], dep["height"])
    offs = synth.offsets_of(specs)
    assert np.array_equal(r0["F"], ref["F"][:, : offs[SPLIT[1]]])
    assert np.array_equal(r1["F"], ref["F"][:, offs[SPLIT[1]]:])


def test_gather_without_process_group_is_local():
    h = np.zeros(3, dtype=exchange.HILL_DTYPE)
    h["height"] = [1.0, 2.0, 3.0]
    out = exchange.gather_hills(h)
    assert np.array_equal(out, h) and out is not h


def test_hill_record_layout_matches_header():
    dt = abp.HILL_DTYPE
    assert dt.itemsize == 48
    assert [dt.fields[k][1] for k in ("s", "height", "step", "walker_id", "pad")] == [0, 24, 32, 40, 44]
