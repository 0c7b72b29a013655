"""Benchmark: bias steps/s of the batched ABP force call on one GB300.

Workload (one "step" of this benchmark = C consecutive MD steps of the whole
hot path a1..a5 for every walker, one launch of the fused kernel):
  64 walkers, each with its own 256 x 256 FP32 grid (value + compensation,
  3 fields), CVs = centre-of-mass distance of two 16-atom groups in
  [0.2, 2.0] nm and a periodic dihedral, sigma = (0.04 nm, 0.1 rad),
  w = 0.5 kJ/mol every 50 steps, gamma = 15; seeded open-loop frames
  (template path + 0.02 nm jitter) resident in HBM, 4000 frames (147 MB,
  larger than L2) cycled.

Reported beside the batched number: the plain one-walker-per-launch form
(three launches per walker per MD step), per-call latency percentiles, an
end-to-end figure through the same public call with host buffers, the
roofline of the fused kernel and the FP64 oracle timed on the host cores.

Multi-GPU (torchrun): every rank runs its own independent 64 walkers
(replicas; no data-path collective), value = all ranks' bias steps / the
slowest rank's time.

--impl reference: the FP64 CPU oracle (oracle/) on the same workload, each
step a bounded sample of MD steps, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bias steps/sec (batched+served vs plain per-walker launch, 1 GB300); p50/p99 latency"
UNIT = "bias steps/s"
NW = 64
NATOMS = 36
FRAMES = 4000
SEED = 2024
# algorithmic bytes per walker-step of this workload (see the design notes):
# coordinates read + forces written as 16-byte records, interpolation corners
# (4 nodes x 3 fields x value+compensation x 4 B), and per deposit the stencil
# read-modify-write (47 x 35 nodes x 3 fields x 2 words x 4 B x 2) plus the
# height's corner read, every 50 steps.
STENCIL_NODES = 47 * 35
NODE_BYTES = 3 * 2 * 4
BYTES_PER_WALKER_STEP = NATOMS * 16 * 2 + 4 * NODE_BYTES + (STENCIL_NODES * NODE_BYTES * 2 + 4 * NODE_BYTES) / 50.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--md-steps", type=int, default=100, help="MD steps per benchmark step (one launch)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tile", default="auto", choices=["auto", "on", "off"])
    ap.add_argument("--group-threads", type=int, default=0)
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(seed):
    from paper_1609_09833_gb300 import synth

    specs = synth.mb64_specs(nw=NW)
    return specs, synth.SweepFrames(NW, seed=seed)


# ---------------------------------------------------------------- reference arm (the oracle)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1609_09833_gb300 import synth

    specs, fr = workload(SEED)
    ws = [oracle.Walker(s) for s in specs]
    fields = [w.new_field() for w in ws]
    per = 5  # MD steps per reference step (a bounded sample of the workload)
    off = synth.offsets_of(specs)
    frames = fr.frames(0, per * (args.warmup + args.steps)).astype(np.float64)
    step = 0
    for _ in range(args.warmup):
        oracle.run(ws, frames[step:step + per], off, step, per, fields=fields, record_forces=False)
        step += per
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(ws, frames[step:step + per], off, step, per, fields=fields, record_forces=False)
        step += per
    dt = time.perf_counter() - t0
    value = NW * per * args.steps / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "64 walkers, own 256x256 grids, COM distance + dihedral, open-loop frames",
                   "md_steps_per_step": per},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per} MD steps x {NW} walkers per step, FP64 C oracle, OpenMP over walkers"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(seconds: float):
    """The oracle as it stands on this host's cores, on a bounded sample."""
    import oracle
    from paper_1609_09833_gb300 import synth

    specs, fr = workload(SEED)
    ws = [oracle.Walker(s) for s in specs]
    fields = [w.new_field() for w in ws]
    off = synth.offsets_of(specs)
    pilot = 40
    frames = fr.frames(0, pilot).astype(np.float64)
    t0 = time.perf_counter()
    oracle.run(ws, frames, off, 0, pilot, fields=fields, record_forces=False)
    per_step = (time.perf_counter() - t0) / pilot
    T = int(max(50, min(20000, seconds / max(per_step, 1e-9))))
    frames = fr.frames(pilot, T).astype(np.float64)
    t0 = time.perf_counter()
    oracle.run(ws, frames, off, pilot, T, fields=fields, record_forces=False)
    dt = time.perf_counter() - t0
    return {"value": NW * T / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"MD steps {pilot}..{pilot + T - 1} of the same 64-walker workload ({NW * T} bias steps, "
                      f"{dt:.1f} s), FP64 C oracle, OpenMP over walkers"}


# ---------------------------------------------------------------- our arm


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    from paper_1609_09833_gb300 import abp, build, synth

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    build.build()
    stream = torch.cuda.current_stream()
    ctx = abp.Context(dev, stream.cuda_stream)
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TILE, {"auto": -1, "on": 1, "off": 0}[args.tile])
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUP_THREADS, args.group_threads)
    specs, fr = workload(SEED + 7919 * rank)
    walkers = ctx.make_walkers(specs)
    C = args.md_steps
    nframes = max(FRAMES // C, 1) * C
    frames = abp.to_records(fr.frames(0, nframes)).cuda()  # [nframes, 64*36, 4]
    A = frames.shape[1]
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    F = torch.zeros(C, A, 4, device="cuda")
    OVER = abp.ABP_FORCES_OVERWRITE
    state = {"md": 0}

    def launch(out=F):
        md = state["md"]
        fi = md % nframes
        if fi + C > nframes:
            fi = 0
        abp.abp_run(ctx.handle, walkers, frames[fi:], abp.ABP_F32, offs, A, out, offs, A, OVER, md, C)
        state["md"] = md + C

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        launch()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            launch()
        e1.record(stream)
        barrier()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    bias_steps = world * NW * C * args.steps
    value = bias_steps / (ms / 1e3)
    kernel_ms = ms / args.steps  # one launch of the fused kernel per step

    # single-MD-step call latency (one launch for all walkers), p50/p99
    lat = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    F1 = torch.zeros(1, A, 4, device="cuda")
    for a, b in ev:
        md = state["md"]
        a.record(stream)
        abp.abp_run(ctx.handle, walkers, frames[md % nframes:], abp.ABP_F32, offs, A, F1, offs, A, OVER, md, 1)
        b.record(stream)
        state["md"] = md + 1
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) * 1e3 for a, b in ev])

    # end to end through the same call with host buffers (pinned), per step:
    # H2D of the step's C frames, the call, D2H of its forces
    host_in = frames[:C].cpu().pin_memory()
    host_out = torch.empty(C, A, 4).pin_memory()
    dev_in = torch.empty_like(frames[:C])
    n_e2e = max(3, min(args.steps, 30))

    def e2e_step():
        md = state["md"]
        dev_in.copy_(host_in, non_blocking=True)
        abp.abp_run(ctx.handle, walkers, dev_in, abp.ABP_F32, offs, A, F, offs, A, OVER, md, C)
        host_out.copy_(F, non_blocking=True)
        state["md"] = md + C

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": NW * C * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(host_in.numel() * 4),
           "d2h_bytes_per_step": int(host_out.numel() * 4)}

    # the plain one-walker-per-launch form on the same workload
    wp = ctx.make_walkers(specs)
    Fp = torch.zeros(A, 4, device="cuda")
    for t in range(3):
        abp.abp_step_plain(ctx.handle, wp, frames[t], abp.ABP_F32, offs, Fp, offs, OVER, t)
    torch.cuda.synchronize()
    n_plain = 20
    t0 = time.perf_counter()
    for t in range(3, 3 + n_plain):
        abp.abp_step_plain(ctx.handle, wp, frames[t], abp.ABP_F32, offs, Fp, offs, OVER, t)
    torch.cuda.synchronize()
    plain_value = NW * n_plain / (time.perf_counter() - t0)

    peaks, src = load_peaks()
    achieved = BYTES_PER_WALKER_STEP * NW * C / (kernel_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "kernel": "k_run<float>", "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs, copy)"
                if src == "measured" else "fallback 6.8 TB/s"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 walkers, own 256x256 FP32+comp grids, COM distance + periodic dihedral, "
                                   "open-loop frames", "md_steps_per_step": C, "walkers_per_gpu": NW,
                       "atoms_per_walker": NATOMS, "grid": "256x256x3 fields", "deposit_stride": 50,
                       "l2": "inputs larger than L2: 4000 resident frames (147 MB) cycled",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps,
            "plain": {"value": plain_value, "unit": UNIT, "ratio": value / plain_value,
                      "form": "3 launches per walker per MD step from a host loop"},
            "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "what": "one MD step of all 64 walkers, one call, CUDA events"},
        }
        print(json.dumps(line), flush=True)
    torch.cuda.synchronize()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
