"""Benchmark: bias steps/s of the batched ABP force call on one GB300.

Headline workload (one "step" of this benchmark = C consecutive closed-loop
MD steps of every walker, one launch of the closed-loop kernel):
  64 walkers, each with its own 256 x 256 FP32 grid (value + compensation,
  3 fields), CVs = centre-of-mass distance of two 16-atom groups in
  [0.2, 2.0] nm and a periodic dihedral, sigma = (0.04 nm, 0.1 rad),
  w = 0.5 kJ/mol every 50 steps, gamma = 15; every atom moves by overdamped
  Langevin dynamics (dt = 0.002 ps, mu = 0.1 nm^2/(kJ/mol ps), kT = 2.5)
  under the bias and the Mueller-Brown surface x 0.1 on the CV box, so each
  step's coordinates come from the previous step's force on the device.
  L2 is flushed before every timed launch (the grids, 134 MB, exceed it
  too).

Reported beside the closed-loop number: the open-loop replay of recorded
frames (the windowed form, 1000-step launches; the method's throughput when
future coordinates are known), the plain one-walker-per-launch form (three
launches per walker per MD step), per-call latency percentiles, an
end-to-end figure through the same public call with host buffers, the
roofline of the kernel and the FP64 oracle timed on the host cores.

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
# Algorithmic bytes per walker-step of the 64-walker workload: the grid
# traffic -- interpolation corners (4 nodes x 3 fields x value +
# compensation x 4 B) and, every 50 steps, the deposit's stencil
# read-modify-write (47 x 35 nodes x 3 fields x 2 words x 4 B, read and
# written) plus the height's corner read -- and the atoms: an open-loop
# replay reads each step's coordinates and writes its forces (36 records of
# 16 B each way); a closed-loop launch keeps the atoms on chip and reads and
# writes them once per launch of C steps.
STENCIL_NODES = 47 * 35
NODE_BYTES = 3 * 2 * 4
GRID_BYTES_PER_WALKER_STEP = 4 * NODE_BYTES + (STENCIL_NODES * NODE_BYTES * 2 + 4 * NODE_BYTES) / 50.0
BYTES_PER_WALKER_STEP = NATOMS * 16 * 2 + GRID_BYTES_PER_WALKER_STEP


def closed_loop_bytes_per_walker_step(C):
    return GRID_BYTES_PER_WALKER_STEP + NATOMS * 16 * 2 / C


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--md-steps", type=int, default=1000, help="MD steps per benchmark step (one launch)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--tile", default="auto", choices=["auto", "on", "off"])
    ap.add_argument("--group-threads", type=int, default=0)
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--only", default=None, choices=["double_well", "uneven", "shared", "serve", "paper_rmsd",
                                                      "headline"],
                    help="run just one of the other workloads (for profiling) and print its record")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """SM clock and clock-event reasons sampled every few ms during the timed
    region (NVML through ctypes; nvidia-smi as a fallback)."""

    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, index: int, period_s: float = 0.005):
        self.index = index
        self.period = period_s
        self.samples = []
        self.max_mhz = None
        self._stop = None
        self._thread = None
        self._nvml = None
        self._smi = None

    def _open_nvml(self):
        import ctypes

        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                lib = None
        if lib is None or lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
            return None
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.max_mhz = float(mx.value)
        getr = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        return lib, h, getr

    def _loop(self):
        import ctypes

        lib, h, getr = self._nvml
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and getr(h, ctypes.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            self._stop.wait(self.period)

    def __enter__(self):
        import threading

        try:
            self._nvml = self._open_nvml()
        except Exception:
            self._nvml = None
        if self._nvml is not None:
            self._stop = threading.Event()
            self._thread = threading.Thread(target=self._loop, daemon=True)
            self._thread.start()
        else:
            try:
                q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                     "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                     "clocks_event_reasons.sw_power_cap")
                self._smi = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                              "--format=csv,noheader,nounits", "-lms", "20"],
                                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                self._smi = None
        return self

    def __exit__(self, *a):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=2)
        if self._smi is not None:
            self._smi.terminate()
            try:
                out, _ = self._smi.communicate(timeout=5)
            except Exception:
                self._smi.kill()
                out, _ = self._smi.communicate()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in out.strip().splitlines():
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 6 and p[0].replace(".", "").isdigit():
                    self.max_mhz = float(p[1]) if p[1].replace(".", "").isdigit() else self.max_mhz
                    bits = sum(1 << i for i in range(4) if p[2 + i].lower() == "active")
                    self.samples.append((float(p[0]), -bits - 1))  # negative: smi-encoded reasons
            self._smi_names = names

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"], "samples": 0}
        sm = [c for c, _ in self.samples]
        reasons = set()
        for _, r in self.samples:
            if r >= 0:
                reasons |= {n for b, n in self.REASONS.items() if r & b}
            else:
                bits = -r - 1
                reasons |= {n for i, n in enumerate(self._smi_names) if bits >> i & 1}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.max_mhz, "reasons": sorted(reasons),
                "samples": len(self.samples), "source": "nvml" if self._nvml is not None else "nvidia-smi"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload(seed):
    from paper_1609_09833_gb300 import synth

    specs = synth.mb64_specs(nw=NW)
    return specs, synth.SweepFrames(NW, seed=seed)


HEADLINE_WORKLOAD = ("64 walkers, own 256x256 FP32+comp grids, COM distance + periodic dihedral, closed loop: "
                     "overdamped Langevin of every atom on the bias + scaled Mueller-Brown surface")


def dynamics(seed):
    """The headline's closed-loop dynamics: Langevin on the scaled
    Mueller-Brown surface mapped to the CV box."""
    from paper_1609_09833_gb300 import synth

    return synth.md_muller_brown(seed=seed, mu=0.1)


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
    md = dynamics(SEED)
    streams = np.arange(NW)
    x = fr.frames(0, 1)[0].astype(np.float64)
    step = 0
    for _ in range(args.warmup):
        x = oracle.md_run(ws, x, off, md, streams, step, per, fields=fields)["x"]
        step += per
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = oracle.md_run(ws, x, off, md, streams, step, per, fields=fields)["x"]
        step += per
    dt = time.perf_counter() - t0
    value = NW * per * args.steps / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD, "md_steps_per_step": per},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per} closed-loop MD steps x {NW} walkers per step, FP64 C oracle, OpenMP "
                                   "over walkers"},
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
    md = dynamics(SEED)
    streams = np.arange(NW)
    pilot = 40
    t0 = time.perf_counter()
    x = oracle.md_run(ws, fr.frames(0, 1)[0].astype(np.float64), off, md, streams, 0, pilot, fields=fields)["x"]
    per_step = (time.perf_counter() - t0) / pilot
    T = int(max(50, min(20000, seconds / max(per_step, 1e-9))))
    t0 = time.perf_counter()
    oracle.md_run(ws, x, off, md, streams, pilot, T, fields=fields)
    dt = time.perf_counter() - t0
    return {"value": NW * T / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"closed-loop MD steps {pilot}..{pilot + T - 1} of the same 64-walker workload ({NW * T} "
                      f"bias steps, {dt:.1f} s), FP64 C oracle, OpenMP over walkers"}


# ---------------------------------------------------------------- the other workloads


def oracle_rate(step_fn, units_per_call, seconds, what):
    """The oracle as it stands on a bounded sample of a workload: one pilot
    call sizes the number of calls to about `seconds` of host time; returns
    the cpu_baseline record (bias steps/s, host threads, the sample)."""
    import oracle

    t0 = time.perf_counter()
    step_fn(0)
    pilot = time.perf_counter() - t0
    n = int(max(1, min(1000, seconds / max(pilot, 1e-9))))
    t0 = time.perf_counter()
    for i in range(n):
        step_fn(1 + i)
    dt = time.perf_counter() - t0
    return {"value": units_per_call * n / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} calls of {what} ({units_per_call * n} bias steps, {dt:.1f} s), FP64 C oracle"}

# Flops of one coordination-number pair as the defined formula has them
# (s = sum 1 / (1 + q^3), q = r^2 / r0^2, and dCN/dx for both atoms):
# differences 3, r^2 5, q 1, q^2 and q^3 2, 1 + q^3 1, the reciprocal 1, the
# sum 1, the gradient factor -6 q^2 sw^2 / r0^2 3, the two 3-vector updates
# 12 (one FMA each, 2 flops) = 29; a minimum image adds d / L and d - L k per
# component, 6 = 35. The ALU rooflines of both CN workloads use these counts.
CN_PAIR_FLOPS = 29
CN_PAIR_FLOPS_PBC = 35


class Fp32Peak:
    """The device's FP32 FMA throughput, measured by the library's FMA kernel
    (abp_fp32_fma_peak) with the SM clock sampled while it runs; the peak at
    another clock scales with the clock."""

    def __init__(self, abp, dev):
        with Clocks(dev) as clk:
            flops, secs = abp.abp_fp32_fma_peak(dev, None, 40000)
        self.tflops = flops / 1e12
        self.seconds = secs
        self.mhz = clk.summary()["sm_mhz"] or 2070.0

    def at(self, sm_mhz):
        return self.tflops * (sm_mhz or self.mhz) / self.mhz

    def source(self, sm_mhz):
        return (f"measured: FMA-chain kernel {self.tflops:.1f} TFLOP/s at {self.mhz:.0f} MHz "
                f"({self.seconds * 1e3:.0f} ms), scaled to {sm_mhz or self.mhz:.0f} MHz")


def _time_loop(torch, fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_double_well(abp, synth, torch, dev):
    """One FP64 walker, COM distance of two 8-atom groups, 512-node grid:
    closed loop on U = 5 (s^2 - 1)^2 (overdamped Langevin, mu = 1, dt =
    0.002, kT = 2.5), and the open-loop replay of a random-walk trajectory."""
    ctx = abp.Context(dev)
    try:
        spec = synth.double_well_com_spec()
        T = 2000
        offs = torch.zeros(1, dtype=torch.int64, device="cuda")
        wc = ctx.make_walkers([spec], precision=abp.ABP_PREC_FP64)
        x = abp.to_records(synth.double_well_com_coords(5)[None], torch.float64).cuda()[0]
        md = synth.md_double_well(seed=5)
        st = {"md": 0}

        def closed():
            abp.abp_md_run(ctx.handle, wc, x, abp.ABP_F64, offs, md, [0], step0=st["md"], nsteps=T)
            st["md"] += T

        ms_closed = _time_loop(torch, closed, 5)
        w = ctx.make_walkers([spec], precision=abp.ABP_PREC_FP64)
        x0 = synth.double_well_com_coords(5)
        frames = x0[None] + np.cumsum(synth.rng(6).normal(scale=0.03, size=(T, 16, 3)), axis=0)
        rec = abp.to_records(frames, torch.float64).cuda()
        F = torch.zeros_like(rec)
        so = {"md": 0}

        def run():
            abp.abp_run(ctx.handle, w, rec, abp.ABP_F64, offs, 16, F, offs, 16, abp.ABP_FORCES_OVERWRITE, so["md"], T)
            so["md"] += T

        ms = _time_loop(torch, run, 5)
        # the plain form on the same frames: three launches per MD step
        wp = ctx.make_walkers([spec], precision=abp.ABP_PREC_FP64)
        for t in range(3):
            abp.abp_step_plain(ctx.handle, wp, rec[t], abp.ABP_F64, offs, F[t], offs, abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        n_plain = 200
        t0 = time.perf_counter()
        for t in range(3, 3 + n_plain):
            abp.abp_step_plain(ctx.handle, wp, rec[t], abp.ABP_F64, offs, F[t], offs, abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        plain = n_plain / (time.perf_counter() - t0)
        import oracle

        ow = [oracle.Walker(spec)]
        ofield = [ow[0].new_field()]
        ox = {"x": x0.astype(np.float64)}

        def ostep(i):
            ox["x"] = oracle.md_run(ow, ox["x"], [0], md, [0], i * 2000, 2000, fields=ofield)["x"]

        cpu = oracle_rate(ostep, 2000, 3.0, "2000 closed-loop MD steps of the walker")
        return {"workload": "1 walker, FP64 end to end, COM distance 2x8 atoms, 512-node grid, stride 100; "
                            "closed loop on U = 5 (s^2-1)^2",
                "value": T / (ms_closed / 1e3), "unit": "bias steps/s", "us_per_step": 1e3 * ms_closed / T,
                "md_steps_per_launch": T, "dtype": "f64", "bound": "latency (one walker's dependent step chain)",
                "open_loop_replay": {"value": T / (ms / 1e3), "us_per_step": 1e3 * ms / T,
                                     "form": "windowed, recorded random-walk frames"},
                "plain": {"value": plain, "form": "3 launches per MD step from a host loop (recorded frames)"},
                "cpu_baseline": cpu}
    finally:
        torch.cuda.synchronize()
        ctx.close()


def bench_paper_rmsd(abp, synth, torch, dev):
    """64 walkers shaped like the paper's ligand runs: two 4-atom RMSD CVs on a
    480 x 480 grid over [0, 12] nm, mABP with compact hills (a = 10 grid
    spacings, p = 20, b = 0.9, c = 0.001), histograms updated every step."""
    ctx = abp.Context(dev)
    try:
        nw, C, chunks = 64, 1000, 4
        specs = synth.paper_rmsd_specs(nw=nw)
        rec = abp.to_records(synth.RmsdFrames(specs, seed=41).frames(0, chunks * C)).cuda()
        A = rec.shape[1]
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        walkers = ctx.make_walkers(specs)
        F = torch.zeros(C, A, 4, device="cuda")
        st = {"md": 0}

        def run():
            fi = (st["md"] // C) % chunks * C
            abp.abp_run(ctx.handle, walkers, rec[fi:], abp.ABP_F32, offs, A, F, offs, A, abp.ABP_FORCES_OVERWRITE,
                        st["md"], C)
            st["md"] += C

        ms = _time_loop(torch, run, 5)
        g = specs[0]["grid"]
        R = [int(math.floor(specs[0]["hill"]["a"][k] / ((g["hi"][k] - g["lo"][k]) / (g["n"][k] - 1)))) for k in
             range(2)]
        box = (2 * R[0] + 1) * (2 * R[1] + 1)
        # coordinates + forces, the look-up node, the stencil read and written every step
        per_step = 8 * 16 * 2 + NODE_BYTES + box * NODE_BYTES * 2
        peaks, src = load_peaks()
        achieved = per_step * nw * C / (ms / 1e3) / 1e9
        import oracle

        ows = [oracle.Walker(sp) for sp in specs]
        ofields = [w.new_field() for w in ows]
        ofr = rec[:200].cpu().numpy()[..., :3].astype(np.float64)
        ooff = synth.offsets_of(specs)

        def ostep(i):
            t = (i * 10) % 190
            oracle.run(ows, ofr[t:t + 10], ooff, i * 10, 10, fields=ofields, record_forces=False)

        cpu = oracle_rate(ostep, nw * 10, 3.0, "10 MD steps of the 64 walkers")
        del ofields
        return {"workload": "64 walkers, 2 RMSD CVs (4 atoms each), 480x480 grid on [0,12] nm, mABP compact hills "
                            "a = 10 spacings, p = 20, b = 0.9, c = 0.001, update every step",
                "value": nw * C / (ms / 1e3), "unit": "bias steps/s", "ms_per_launch": ms, "md_steps_per_launch": C,
                "stencil_nodes": box,
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": achieved / peaks["hbm_gbs"], "bytes_per_walker_step": per_step,
                             "kernel": "k_win<float> (windowed form)", "peak_source": src},
                "cpu_baseline": cpu}
    finally:
        torch.cuda.synchronize()
        ctx.close()


def bench_uneven(abp, synth, torch, dev, sm_mhz, fp32):
    """1000 walkers: 40 % 1D / 50 % 2D / 10 % 3D grids, CN 40 x 400 each."""
    from paper_1609_09833_gb300 import autotune

    ctx = abp.Context(dev)
    try:
        nw, C = 1000, 25
        specs = synth.uneven1000_specs(seed=31, nw=nw)
        tm = synth.uneven1000_templates(31, nw=nw)
        rec = abp.to_records(synth.JitterFrames(tm, seed=32).frames(0, C)).cuda()
        A = rec.shape[1]
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        tuned = autotune.tune(ctx, specs, rec, offs, C)
        walkers = ctx.make_walkers(specs)
        F = torch.zeros_like(rec)
        st = {"md": 0}

        def run():
            abp.abp_run(ctx.handle, walkers, rec, abp.ABP_F32, offs, A, F, offs, A, abp.ABP_FORCES_OVERWRITE,
                        st["md"], C)
            st["md"] += C

        ms = _time_loop(torch, run, 6)
        flops = nw * C * 40 * 400 * CN_PAIR_FLOPS
        achieved = flops / (ms / 1e3) / 1e12
        peak = fp32.at(sm_mhz)
        # the same launch replayed from a CUDA graph
        s = torch.cuda.Stream()
        ctx.set_stream(s.cuda_stream)
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            abp.abp_run(ctx.handle, walkers, rec, abp.ABP_F32, offs, A, F, offs, A, abp.ABP_FORCES_OVERWRITE,
                        10 ** 6, C)
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ms_graph = _time_loop(torch, g.replay, 6)
        # the plain form: three launches per walker per MD step
        wp = ctx.make_walkers(specs)
        Fp = torch.zeros_like(rec[0])
        abp.abp_step_plain(ctx.handle, wp, rec[0], abp.ABP_F32, offs, Fp, offs, abp.ABP_FORCES_OVERWRITE, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(1, 3):
            abp.abp_step_plain(ctx.handle, wp, rec[t], abp.ABP_F32, offs, Fp, offs, abp.ABP_FORCES_OVERWRITE, t)
        torch.cuda.synchronize()
        plain = nw * 2 / (time.perf_counter() - t0)
        import oracle

        ns = 100
        ows = [oracle.Walker(sp) for sp in specs[:ns]]
        ofields = [w.new_field() for w in ows]
        ofr = rec[:, :synth.offsets_of(specs)[ns]].cpu().numpy()[..., :3].astype(np.float64)
        ooff = synth.offsets_of(specs[:ns])

        def ostep(i):
            t = i % C
            oracle.run(ows, ofr[t:t + 1], ooff, i, 1, fields=ofields, record_forces=False)

        cpu = oracle_rate(ostep, ns, 3.0, f"one MD step of the first {ns} walkers")
        return {"workload": "1000 walkers (40% 1D 1024, 50% 2D 128^2/256^2/512^2, 10% 3D 64^3), CN 40x400, "
                            "jitter frames, one launch per 25 MD steps",
                "value": nw * C / (ms / 1e3), "unit": "bias steps/s", "ms_per_launch": ms,
                "graph_replay": {"value": nw * C / (ms_graph / 1e3), "ms_per_launch": ms_graph},
                "plain": {"value": plain, "ratio": nw * C / (ms / 1e3) / plain,
                          "form": "3 launches per walker per MD step from a host loop"},
                "cpu_baseline": cpu,
                "tuned": tuned["best"],
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "kernel": "k_run / k_run_lean (per-step form, CN pairs)",
                             "traffic": captured_traffic("k_run_uneven1000", nw * C),
                             "flops_per_pair": CN_PAIR_FLOPS, "peak_source": fp32.source(sm_mhz)}}
    finally:
        torch.cuda.synchronize()
        ctx.close()


def bench_shared(abp, synth, torch, dev, sm_mhz, fp32):
    """32 walkers on one shared 256^3 grid, 200 x 10,000-atom CN each: the
    closed loop (free overdamped Langevin of every atom under the bias, the
    phased form's five launches plus the move per MD step), replayed as a
    CUDA graph of C steps; the open-loop replay of jitter frames beside it;
    the pair kernel's own time from the library's per-kernel timing."""
    ctx = abp.Context(dev)
    try:
        nw, C = 32, 10
        specs = synth.shared256_specs(nw=nw)
        tm = synth.shared256_templates(41, nw=nw)
        rec = abp.to_records(synth.JitterFrames(tm, seed=42).frames(0, C)).cuda()
        A = rec.shape[1]
        offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
        md = synth.md_params(seed=43, mu=0.05)
        streams = np.arange(nw)
        # closed loop
        wc = ctx.make_walkers(specs)
        x = rec[0].clone()
        abp.abp_deposit_log_enable(ctx.handle, 1 << 16)
        st = {"md": 0}

        def closed():
            abp.abp_md_run(ctx.handle, wc, x, abp.ABP_F32, offs, md, streams, step0=st["md"], nsteps=C)
            st["md"] += C

        ms_direct = _time_loop(torch, closed, 3)
        s = torch.cuda.Stream()
        ctx.set_stream(s.cuda_stream)
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            abp.abp_md_run(ctx.handle, wc, x, abp.ABP_F32, offs, md, streams, step0=10 ** 6, nsteps=C)
        ctx.set_stream(torch.cuda.current_stream().cuda_stream)
        ms_graph = _time_loop(torch, g.replay, 5)
        log = abp.abp_deposit_log_readout(ctx.handle, 1 << 16)
        # the pair kernel's own time, direct calls with per-kernel timing
        abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TIMING, 1)
        abp.abp_kernel_times(ctx.handle)
        for _ in range(3):
            closed()
        times = abp.abp_kernel_times(ctx.handle)
        abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TIMING, 0)
        n_cn, ms_cn_total = times.get("k_big_cn", (0, float("nan")))
        ms_cn = ms_cn_total / max(n_cn, 1)
        step_ms = sum(v[1] for v in times.values()) / max(n_cn, 1)
        flops_launch = nw * 200 * 10_000 * CN_PAIR_FLOPS_PBC
        achieved = flops_launch / (ms_cn / 1e3) / 1e12
        peak = fp32.at(sm_mhz)
        # the open loop on jitter frames (the same walkers' shape)
        wo = ctx.make_walkers(specs)
        F = torch.zeros_like(rec)
        so = {"md": 0}

        def run():
            abp.abp_run(ctx.handle, wo, rec, abp.ABP_F32, offs, A, F, offs, A, abp.ABP_FORCES_OVERWRITE,
                        so["md"], C)
            so["md"] += C

        ms_open = _time_loop(torch, run, 3)
        import oracle

        ows = [oracle.Walker(sp) for sp in specs]
        oshared = ows[0].new_field()
        ofr = rec.cpu().numpy()[..., :3].astype(np.float64)
        ooff = synth.offsets_of(specs)

        def ostep(i):
            t = i % C
            oracle.run(ows, ofr[t:t + 1], ooff, i, 1, fields=[oshared] * nw, record_forces=False)

        cpu = oracle_rate(ostep, nw, 3.0, "one MD step of the 32 walkers on the shared grid")
        del oshared
        overlap = None
        if len(log["step"]):
            st0 = log["step"][0]
            ic = log["ic"][log["step"] == st0]
            R = 8
            pairs = sum(1 for a in range(len(ic)) for b2 in range(a + 1, len(ic))
                        if np.all(np.abs(ic[a] - ic[b2]) <= 2 * R))
            overlap = {"hills_per_deposit_step": int(len(ic)), "overlapping_box_pairs": int(pairs)}
        return {"workload": "32 walkers, one shared 256^3 grid (FP64 shadow), 200 ligand + 10,000 environment "
                            "atoms, 6 nm periodic box, stride 10; closed loop (free overdamped Langevin, mu = 0.05), "
                            "10 MD steps per call, CUDA-graph replay",
                "value": nw * C / (ms_graph / 1e3), "unit": "bias steps/s", "ms_per_md_step": ms_graph / C,
                "value_direct_calls": nw * C / (ms_direct / 1e3), "gpu_launches_per_md_step": 6,
                "open_loop_replay": {"value": nw * C / (ms_open / 1e3), "gpu_launches_per_md_step": 5},
                "kernel_ms_per_md_step": {k: v[1] / max(v[0], 1) for k, v in times.items()},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "kernel": "k_big_cn (pair kernel), its own CUDA-event time",
                             "traffic": captured_traffic("k_big_cn_shared256", nw),
                             "kernel_share_of_step": ms_cn / step_ms if step_ms > 0 else None,
                             "flops_per_pair": CN_PAIR_FLOPS_PBC, "peak_source": fp32.source(sm_mhz)},
                "cpu_baseline": cpu,
                "deposit_contention": overlap}
    finally:
        torch.cuda.synchronize()
        ctx.close()


def bench_serve(abp, synth, torch, dev, seconds=2.0, rate=20_000.0):
    """4096 simulations (2D grids 64^2..1024^2, 8..256 atoms, stride 20..500):
    Poisson step requests at `rate`/s for `seconds` (latency), then a deep
    backlog (saturation throughput)."""
    import threading

    ctx = abp.Context(dev, budget=120 << 30)
    srv = None
    try:
        nsim = 4096
        specs = synth.serve_specs(seed=61, nsim=nsim)
        tmpl = synth.serve_templates(61, specs)
        srv = abp.abp_server_create(ctx.handle, max_batch=4096, max_atoms=256, nstreams=2)
        sims, keep = [], []
        for sp in specs:
            desc, k = abp.walker_desc(sp)
            keep.append(k)
            sims.append(abp.abp_server_admit(srv, abp.grid_desc(sp["grid"]), desc))
        hbm = abp.abp_ctx_bytes(ctx.handle)[0]
        r = synth.rng(62)
        nf = 4
        frames = []
        for t in tmpl:
            x = np.zeros((nf, t.shape[0], 4), dtype=np.float32)
            x[..., :3] = t[None] + r.normal(scale=0.02, size=(nf,) + t.shape)
            frames.append(x)
        forces = [np.zeros_like(f[0]) for f in frames]
        step = np.zeros(nsim, dtype=np.int64)
        results = []
        done = threading.Event()

        def poller():
            while not done.is_set():
                results.extend(abp.abp_server_poll(srv, 8192, wait_ms=20))
            results.extend(abp.abp_server_poll(srv, 1 << 20))

        # warm-up: one request per simulation
        th = threading.Thread(target=poller)
        th.start()
        for i in range(nsim):
            abp.abp_server_submit(srv, sims[i], int(step[i]), frames[i][0], forces[i], i)
            step[i] += 1
        while len(results) < nsim:
            time.sleep(0.01)
        results.clear()
        # Poisson arrivals
        n_req = int(rate * seconds)
        gaps = r.exponential(1.0 / rate, size=n_req)
        who = r.integers(0, nsim, size=n_req)
        t0 = time.perf_counter()
        t_next = t0
        for k in range(n_req):
            t_next += gaps[k]
            while time.perf_counter() < t_next:
                pass
            i = int(who[k])
            abp.abp_server_submit(srv, sims[i], int(step[i]), frames[i][step[i] % nf], forces[i], i)
            step[i] += 1
        t_sub = time.perf_counter() - t0
        while len(results) < n_req and time.perf_counter() - t0 < seconds + 30:
            time.sleep(0.005)
        t_all = time.perf_counter() - t0
        lat = np.array([x.t_done - x.t_submit for x in results]) * 1e6
        batches = np.array([x.batch for x in results])
        poisson = {"offered_rate": rate, "requests": n_req, "completed": len(results),
                   "achieved_rate": len(results) / t_all, "submit_rate": n_req / t_sub,
                   "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                   "mean_batch": float(batches.mean())}
        results.clear()
        # saturation: a backlog of `depth` requests per simulation, queued in
        # one call; five repeats, the median reported with the spread. The
        # throughput is taken on the server's clock: from the submit call to
        # the moment the last forces were in the caller's buffer
        # (abp_result.t_submit / t_done), so the Python poller's wake-ups do
        # not enter it; the wall-clock figure seen from Python is kept beside.
        depth = 16
        reps = []
        tw0 = None
        for rep in range(6):  # the first is a warm-up (its slabs are allocated and faulted in)
            if rep == 1:
                reps.clear()
                tw0 = abp.abp_server_times(srv)
            results.clear()
            order = [i for d in range(depth) for i in range(nsim)]
            sim_ids = np.array([sims[i] for i in order], dtype=np.int64)
            steps_arr = np.empty(len(order), dtype=np.int64)
            chunks = []
            for k, i in enumerate(order):
                steps_arr[k] = step[i]
                chunks.append(frames[i][step[i] % nf])
                step[i] += 1
            packed = np.ascontiguousarray(np.concatenate(chunks, axis=0))
            out = np.zeros_like(packed)
            t0 = time.perf_counter()
            abp.abp_server_submit_many(srv, sim_ids, steps_arr, packed, out)
            t_sub = time.perf_counter() - t0
            while len(results) < nsim * depth and time.perf_counter() - t0 < 120:
                time.sleep(0.002)
            t_all = time.perf_counter() - t0
            span = max(x.t_done for x in results) - min(x.t_submit for x in results)
            reps.append({"completed": len(results), "throughput": len(results) / span,
                         "throughput_wall": len(results) / t_all, "submit_seconds": t_sub,
                         "mean_batch": float(np.mean([x.batch for x in results]))})
        tw1 = abp.abp_server_times(srv)
        tput = sorted(r["throughput"] for r in reps)
        med = tput[len(tput) // 2]
        sat = {"requests_per_repeat": nsim * depth, "repeats": reps, "throughput": med,
               "spread": (tput[-1] - tput[0]) / med,
               "clock": "server steady clock, submit to the last forces delivered",
               "worker_seconds": {k: tw1[k] - tw0[k] for k in tw0}}
        done.set()
        th.join()
        # the plain form on the same simulations' shapes: 256 of them as
        # walkers of their own, three launches per walker per MD step
        pctx = abp.Context(dev)
        try:
            np_ = 256
            psp = specs[:np_]
            pw = pctx.make_walkers(psp)
            xs = np.concatenate([frames[i][0][:, :3] for i in range(np_)])
            prec = abp.to_records(xs[None]).cuda()[0]
            poffs = torch.tensor(synth.offsets_of(psp), dtype=torch.int64, device="cuda")
            pF = torch.zeros_like(prec)
            for t in range(2):
                abp.abp_step_plain(pctx.handle, pw, prec, abp.ABP_F32, poffs, pF, poffs, abp.ABP_FORCES_OVERWRITE, t)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n_plain = 5
            for t in range(2, 2 + n_plain):
                abp.abp_step_plain(pctx.handle, pw, prec, abp.ABP_F32, poffs, pF, poffs, abp.ABP_FORCES_OVERWRITE, t)
            torch.cuda.synchronize()
            plain = np_ * n_plain / (time.perf_counter() - t0)
        finally:
            pctx.close()
        import oracle

        ns = 32
        ows = [oracle.Walker(sp) for sp in specs[:ns]]
        ofields = [w.new_field() for w in ows]
        ofr = np.concatenate([frames[i][:, :, :3] for i in range(ns)], axis=1).astype(np.float64)
        ooff = synth.offsets_of(specs[:ns])

        def ostep(i):
            t = i % nf
            oracle.run(ows, ofr[t:t + 1], ooff, i, 1, fields=ofields, record_forces=False)

        cpu = oracle_rate(ostep, ns, 3.0, f"one step of {ns} of the simulations")
        del ofields
        st = abp.abp_server_stats(srv)
        return {"workload": "4096 simulations, 2D grids 64^2..1024^2 FP32+comp, 8..256 atoms, stride 20..500; "
                            "Poisson step requests (host coords in, host forces out)",
                "value": sat["throughput"], "unit": "bias steps/s (served, saturated; median of 5)",
                "admitted": len(sims), "hbm_bytes": hbm, "poisson": poisson, "saturation": sat,
                "plain": {"value": plain, "ratio": sat["throughput"] / plain,
                          "form": "256 of the simulations as plain-form walkers, 3 launches per walker per step"},
                "cpu_baseline": cpu,
                "launches": st["launches"]}
    finally:
        if srv is not None:
            abp.abp_server_destroy(srv)
        torch.cuda.synchronize()
        ctx.close()


# ---------------------------------------------------------------- our arm


# The device sources each captured kernel is compiled from (its own file and
# the headers it includes): a capture stays valid while these are unchanged.
KERNEL_SOURCES = {
    "k_md_mb64": ["abp_md.cu", "abp_md.cuh", "abp_window_ops.cuh", "abp_device.cuh", "abp_internal.cuh",
                  "abp_launch.h"],
    "k_win_mb64": ["abp_kernels.cu", "abp_window_ops.cuh", "abp_device.cuh", "abp_internal.cuh", "abp_launch.h"],
    "k_run_uneven1000": ["abp_kernels.cu", "abp_window_ops.cuh", "abp_device.cuh", "abp_internal.cuh",
                         "abp_launch.h"],
    "k_big_cn_shared256": ["abp_big.cu", "abp_md.cuh", "abp_device.cuh", "abp_internal.cuh", "abp_launch.h"],
}


def kernel_source_hash(kernel_key):
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1609_09833_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES[kernel_key]):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel_key, units_per_launch):
    """DRAM bytes per launch from the committed ncu capture, scaled to this
    launch's units, or None when the kernel's sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel_key]
    except (OSError, ValueError, KeyError):
        return None
    if rec.get("source_hash") != kernel_source_hash(kernel_key):
        return None
    return rec["dram_bytes"] / rec["units"] * units_per_launch


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    from paper_1609_09833_gb300 import abp, build, synth

    if args.only == "headline":  # the headline line alone (profiling runs)
        args.only, args.no_extra, args.no_cpu_baseline = None, True, True
    if args.only:
        torch.cuda.set_device(0)
        build.build()
        fn = {"double_well": lambda: bench_double_well(abp, synth, torch, 0),
              "uneven": lambda: bench_uneven(abp, synth, torch, 0, 2070.0, Fp32Peak(abp, 0)),
              "shared": lambda: bench_shared(abp, synth, torch, 0, 2070.0, Fp32Peak(abp, 0)),
              "serve": lambda: bench_serve(abp, synth, torch, 0),
              "paper_rmsd": lambda: bench_paper_rmsd(abp, synth, torch, 0)}[args.only]
        print(json.dumps({"only": args.only, **fn()}), flush=True)
        return 0

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
    md = dynamics(SEED + rank)
    streams = np.arange(NW) + NW * rank
    C = args.md_steps
    A = NW * NATOMS
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    x0 = abp.to_records(fr.frames(0, 1)).cuda()[0]  # [64*36, 4]: the walkers' atoms at step 0
    x = x0.clone()
    walkers = ctx.make_walkers(specs)
    OVER = abp.ABP_FORCES_OVERWRITE
    state = {"md": 0}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # twice L2

    def launch():
        md0 = state["md"]
        abp.abp_md_run(ctx.handle, walkers, x, abp.ABP_F32, offs, md, streams, step0=md0, nsteps=C)
        state["md"] = md0 + C

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        launch()
    barrier()
    # each timed launch starts with L2 flushed (the flush itself untimed)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(dev) as clk:
        barrier()
        for a, b in ev:
            flush.fill_(1)
            a.record(stream)
            launch()
            b.record(stream)
        barrier()
    ms = float(sum(a.elapsed_time(b) for a, b in ev))
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    bias_steps = world * NW * C * args.steps
    value = bias_steps / (ms / 1e3)
    kernel_ms = ms / args.steps  # one launch of the closed-loop kernel per step

    # one MD step of all 64 walkers per call (a host-coupled MD step), p50/p99;
    # the call's arguments marshalled once, as an engine holds them
    wa, mdd, sa = abp.walker_array(walkers), abp.md_desc(md), np.ascontiguousarray(streams, dtype=np.uint32)
    evl = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    for a, b in evl:
        md0 = state["md"]
        a.record(stream)
        abp.abp_md_run(ctx.handle, wa, x, abp.ABP_F32, offs, mdd, sa, step0=md0, nsteps=1)
        b.record(stream)
        state["md"] = md0 + 1
    torch.cuda.synchronize()
    lat = np.array([a.elapsed_time(b) * 1e3 for a, b in evl])
    # one MD step per call, as a host MD engine calls it: back-to-back calls
    # (launch overhead included; the call's arguments marshalled once, as an
    # engine holds them) and the same calls replayed from a CUDA graph
    n1 = 200
    t0 = time.perf_counter()
    for _ in range(n1):
        md0 = state["md"]
        abp.abp_md_run(ctx.handle, wa, x, abp.ABP_F32, offs, mdd, sa, step0=md0, nsteps=1)
        state["md"] = md0 + 1
    torch.cuda.synchronize()
    one_step = NW * n1 / (time.perf_counter() - t0)
    gs = torch.cuda.Stream()
    ctx.set_stream(gs.cuda_stream)
    g1 = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g1, stream=gs):
        for k in range(50):
            abp.abp_md_run(ctx.handle, walkers, x, abp.ABP_F32, offs, md, streams, step0=10 ** 7 + k, nsteps=1)
    ctx.set_stream(stream.cuda_stream)
    ms_g1 = _time_loop(torch, g1.replay, 5)
    one_step_graph = NW * 50 / (ms_g1 / 1e3)

    # end to end through the same call with host buffers (pinned), per step:
    # H2D of the walkers' atoms, C closed-loop steps, D2H of the moved atoms
    host_in = x.cpu().pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    n_e2e = max(3, min(args.steps, 30))

    def e2e_step():
        md0 = state["md"]
        x.copy_(host_in, non_blocking=True)
        abp.abp_md_run(ctx.handle, walkers, x, abp.ABP_F32, offs, md, streams, step0=md0, nsteps=C)
        host_out.copy_(x, non_blocking=True)
        state["md"] = md0 + C

    for _ in range(2):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": NW * C * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(host_in.numel() * 4),
           "d2h_bytes_per_step": int(host_out.numel() * 4),
           "what": f"per benchmark step: the {NW} walkers' atoms from pinned host memory, one {C}-step closed-loop "
                   "call, the moved atoms back to pinned host memory; host clock, no L2 flush between steps"}

    # the open-loop replay of recorded frames (windowed form, the former
    # headline) and the plain one-walker-per-launch form on those frames
    nframes = max(FRAMES // C, 1) * C
    frames = abp.to_records(fr.frames(0, nframes)).cuda()  # [nframes, 64*36, 4], larger than L2
    tuned = None
    if args.tile == "auto" and args.group_threads == 0:
        from paper_1609_09833_gb300 import autotune

        tuned = autotune.tune(ctx, specs, frames[:C], offs, C)["best"]
    wo = ctx.make_walkers(specs)
    F = torch.zeros(C, A, 4, device="cuda")
    so = {"md": 0}

    def launch_open():
        md0 = so["md"]
        fi = md0 % nframes
        if fi + C > nframes:
            fi = 0
        abp.abp_run(ctx.handle, wo, frames[fi:], abp.ABP_F32, offs, A, F, offs, A, OVER, md0, C)
        so["md"] = md0 + C

    for _ in range(3):
        launch_open()
    torch.cuda.synchronize()
    n_open = max(10, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_open):
        launch_open()
    e1.record(stream)
    torch.cuda.synchronize()
    open_ms = e0.elapsed_time(e1) / n_open
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
    psrc = f"{src} (MEASURED_PEAKS.json hbm_gbs, copy)" if src == "measured" else "fallback 6.8 TB/s"
    cl_bytes = closed_loop_bytes_per_walker_step(C)
    achieved = cl_bytes * NW * C / (kernel_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": captured_traffic("k_md_mb64", NW * C),
                "kernel": "k_md<float, 2> (closed-loop form, a group of 4 warps per walker)", "peak_source": psrc,
                "bytes_per_walker_step": cl_bytes,
                "limiter": "each walker's steps form a dependent chain (CVs, grid corners from L2, force, move); "
                           "64 chains on 64 SMs",
                "us_per_walker_step": 1e3 * kernel_ms / C}
    open_achieved = BYTES_PER_WALKER_STEP * NW * C / (open_ms / 1e3) / 1e9
    open_loop = {"workload": "the same 64 walkers replaying 4000 recorded open-loop frames (147 MB, larger than "
                             "L2, cycled), windowed form", "value": NW * C / (open_ms / 1e3), "unit": UNIT,
                 "ms_per_launch": open_ms, "md_steps_per_launch": C, "launch_shape": tuned,
                 "roofline": {"bound": "hbm", "achieved": open_achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": open_achieved / peaks["hbm_gbs"],
                              "traffic": captured_traffic("k_win_mb64", NW * C),
                              "kernel": "k_win<float> (windowed form)", "peak_source": psrc,
                              "bytes_per_walker_step": BYTES_PER_WALKER_STEP}}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
    clocks = clk.summary()
    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        sm = clocks["sm_mhz"] or 2070.0
        fp32 = Fp32Peak(abp, dev)
        extra = {"open_loop_replay64": open_loop,
                 "fp32_peak": {"tflops": fp32.tflops, "sm_mhz": fp32.mhz, "seconds": fp32.seconds,
                               "how": "abp_fp32_fma_peak: 8 x SMs CTAs x 256 threads x 8 FMA chains"}}
        for name, fn in (("double_well_fp64", lambda: bench_double_well(abp, synth, torch, dev)),
                         ("uneven1000", lambda: bench_uneven(abp, synth, torch, dev, sm, fp32)),
                         ("shared256", lambda: bench_shared(abp, synth, torch, dev, sm, fp32)),
                         ("serve4096", lambda: bench_serve(abp, synth, torch, dev)),
                         ("paper_rmsd_mabp64", lambda: bench_paper_rmsd(abp, synth, torch, dev))):
            try:
                extra[name] = fn()
            except Exception as e:  # report, do not hide the headline
                extra[name] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": HEADLINE_WORKLOAD, "md_steps_per_step": C, "walkers_per_gpu": NW,
                       "atoms_per_walker": NATOMS, "grid": "256x256x3 fields", "deposit_stride": 50,
                       "dynamics": "overdamped Langevin, dt 0.002 ps, mu 0.1, kT 2.5, Mueller-Brown x 0.1",
                       "l2": "flushed before every timed launch (256 MB write); grids 134 MB",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps,
            "plain": {"value": plain_value, "unit": UNIT, "ratio": value / plain_value,
                      "form": "3 launches per walker per MD step from a host loop (open-loop frames)"},
            "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "what": "one closed-loop MD step of all 64 walkers, one call, CUDA events"},
            "one_step_per_call": {"value": one_step, "graph_replay": one_step_graph, "unit": UNIT,
                                  "ratio_to_plain": one_step / plain_value,
                                  "what": "the same walkers, one closed-loop MD step of all 64 per call (as a host MD "
                                          "engine calls the bias), back to back; and 50 such calls in a CUDA graph"},
            "other_workloads": extra,
        }
        print(json.dumps(line), flush=True)
    torch.cuda.synchronize()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
