"""Small runs of every form of the library, for the checked-build test.

Run as `python -m tests.checked_workloads OUT.npz` with ABP_LIBRARY naming
the library to load (the checked or the normal build): it runs the windowed
form (WT and mABP), the per-step fused form (coordination numbers, 1D to 3D
grids), the phased form on a shared grid, the closed loop (fused and
phased), the plain form, the allocation-free step and the server, saves
every force array and grid to OUT.npz, and prints one JSON line with the
count of out-of-grid node indices the library saw and whether it is the
checked build.
"""
import json
import sys

import numpy as np
import torch

from paper_1609_09833_gb300 import abp, synth


def _replay(ctx, specs, frames, chunks=1, prec=abp.ABP_PREC_FP32_COMP):
    walkers = ctx.make_walkers(specs, precision=prec)
    rec = abp.to_records(frames).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    F = torch.zeros_like(rec)
    T, A = rec.shape[0], rec.shape[1]
    bounds = np.linspace(0, T, chunks + 1).astype(int)
    for a, b in zip(bounds[:-1], bounds[1:]):
        abp.abp_run(ctx.handle, walkers, rec[a:], abp.ABP_F32, offs, A, F[a:], offs, A, abp.ABP_FORCES_OVERWRITE,
                    int(a), int(b - a))
    torch.cuda.synchronize()
    return F.cpu().numpy(), [ctx.bias(w) for w in walkers]


def _mabp(specs, a_bins=8.0, c=0.2, stride=2):
    out = []
    for sp in specs:
        sp = dict(sp)
        g = sp["grid"]
        a = [synth.bins(g, k, a_bins) for k in range(len(g["n"]))]
        sp["hill"] = synth.mabp_hill(a, 20, 0.9, c, kT=2.5, stride=stride, w=1.0)
        out.append(sp)
    return out


def main(path):
    torch.cuda.set_device(0)
    abp.load()
    ctx = abp.Context(0)
    out = {}
    # windowed form, WT (hills crossing the periodic seam) and mABP
    specs = synth.mb64_specs(nw=4, stride=5)
    fr = synth.SweepFrames(4, seed=5, period=(150, 400), dihedral_period=(100, 300)).frames(0, 120)
    F, B = _replay(ctx, specs, fr, chunks=2)
    out["win_F"] = F
    out.update({f"win_B{i}": b for i, b in enumerate(B)})
    F, B = _replay(ctx, _mabp(synth.mb64_specs(nw=3, stride=2)), fr[:, :108], chunks=2)
    out["mabp_F"] = F
    out.update({f"mabp_B{i}": b for i, b in enumerate(B)})
    # per-step fused form, coordination numbers on 1D, 2D and 3D grids
    specs = synth.uneven1000_specs(seed=3, nw=12, stride=10, sizes_2d=(48, 64), n1d=256, n3d=24)
    fr = synth.JitterFrames(synth.uneven1000_templates(3, nw=12), seed=4).frames(0, 30)
    F, B = _replay(ctx, specs, fr)
    out["run_F"] = F
    out.update({f"run_B{i}": b for i, b in enumerate(B)})
    # phased form on a shared grid
    specs = synth.shared256_specs(nw=4, n=32, n_lig=16, n_env=200, box=3.0, stride=2, cn_range=(30.0, 130.0))
    fr = synth.JitterFrames(synth.shared256_templates(11, nw=4, n_lig=16, n_env=200, box=3.0), seed=12).frames(0, 6)
    F, B = _replay(ctx, specs, fr)
    out["big_F"] = F
    out["big_B"] = B[0]
    # closed loop: the fused form and the phased form
    specs = synth.mb64_specs(nw=4, stride=3)
    ws = ctx.make_walkers(specs)
    x = abp.to_records(synth.SweepFrames(4, seed=29).frames(0, 1)[0][None]).cuda()[0]
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    abp.abp_md_run(ctx.handle, ws, x, abp.ABP_F32, offs, synth.md_muller_brown(seed=7), np.arange(4), step0=0, nsteps=40)
    torch.cuda.synchronize()
    out["md_x"] = x.cpu().numpy()
    out.update({f"md_B{i}": ctx.bias(w) for i, w in enumerate(ws)})
    specs = synth.shared256_specs(nw=3, n=32, n_lig=16, n_env=200, box=3.0, stride=2, cn_range=(30.0, 130.0))
    for sp in specs:
        sp["shared"] = "md"
    ws = ctx.make_walkers(specs)
    x0 = np.concatenate(synth.shared256_templates(13, nw=3, n_lig=16, n_env=200, box=3.0)).astype(np.float32)
    x = abp.to_records(x0[None]).cuda()[0]
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    abp.abp_md_run(ctx.handle, ws, x, abp.ABP_F32, offs, synth.md_params(seed=3, mu=0.05), np.arange(3), step0=0,
                   nsteps=8)
    torch.cuda.synchronize()
    out["mdbig_x"] = x.cpu().numpy()
    # plain form
    specs = synth.mb64_specs(nw=2, stride=2)
    wp = ctx.make_walkers(specs)
    fr = synth.SweepFrames(2, seed=9).frames(0, 6)
    rec = abp.to_records(fr).cuda()
    offs = torch.tensor(synth.offsets_of(specs), dtype=torch.int64, device="cuda")
    Fp = torch.zeros_like(rec)
    for t in range(6):
        abp.abp_step_plain(ctx.handle, wp, rec[t], abp.ABP_F32, offs, Fp[t], offs, abp.ABP_FORCES_OVERWRITE, t)
    torch.cuda.synchronize()
    out["plain_F"] = Fp.cpu().numpy()
    # the allocation-free step (its grid is the caller's)
    spec = synth.mb64_specs(nw=1, stride=1)[0]
    grid = torch.zeros(int(np.prod(spec["grid"]["n"])), 8, device="cuda")
    wdesc, keep = abp.walker_desc(spec)
    Fs = torch.zeros(2, spec["natoms"], 4, device="cuda")
    for t in range(2):
        abp.abp_step_static(0, torch.cuda.current_stream().cuda_stream, abp.grid_desc(spec["grid"]), grid, wdesc,
                            rec[t, :spec["natoms"]].contiguous(), abp.ABP_F32, Fs[t], abp.ABP_FORCES_OVERWRITE, t)
    torch.cuda.synchronize()
    out["static_F"] = Fs.cpu().numpy()
    out["static_grid"] = grid.cpu().numpy()
    # the server
    srv = abp.abp_server_create(ctx.handle, max_batch=16, max_atoms=256, nstreams=2)
    try:
        sspecs = synth.serve_specs(seed=3, nsim=6, side=(64, 160), stride=(2, 5))
        tm = synth.serve_templates(3, sspecs)
        sims, keeps = [], []
        for sp in sspecs:
            d, k = abp.walker_desc(sp)
            keeps.append(k)
            sims.append(abp.abp_server_admit(srv, abp.grid_desc(sp["grid"]), d))
        r = synth.rng(5)
        outs = []
        for t in range(5):
            for i, s in enumerate(sims):
                xr = np.zeros((tm[i].shape[0], 4), dtype=np.float32)
                xr[:, :3] = tm[i] + r.normal(scale=0.02, size=tm[i].shape)
                f = np.zeros_like(xr)
                outs.append(f)
                abp.abp_server_submit(srv, s, t, xr, f)
        got, tries = [], 0
        while len(got) < len(outs) and tries < 1200:
            got += abp.abp_server_poll(srv, 256, wait_ms=50)
            tries += 1
        assert len(got) == len(outs)
        assert all(g.status == 0 for g in got)
        out["serve_F"] = np.concatenate(outs)
    finally:
        abp.abp_server_destroy(srv)
    n, checked = abp.abp_checked_violations(ctx.handle)
    ctx.close()
    np.savez(path, **out)
    print(json.dumps({"violations": n, "checked": checked}))


if __name__ == "__main__":
    main(sys.argv[1])
