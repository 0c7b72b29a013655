"""Walkers on several GPUs that share one bias: hill exchange.

In a multiple-walker run every walker adds its hills to one common bias
grid. Spread over ranks, each rank keeps a full replica of the shared grid
and advances only its own walkers. One MD step is then:

1. ``hills``: the rank's walkers evaluate their CVs and their well-tempered
   hill heights (text after Eq. (Cupdate)) from the replica as it stood
   before the step's deposits and return their hill records, without
   depositing (``abp_shared_hills``);
2. ``gather_hills``: the records of all ranks are all-gathered and
   concatenated in rank order (within a rank, in walker order), so every rank
   holds the same list: the walkers' global order;
3. ``apply``: every rank deposits the whole list into its replica in that
   order (Eq. (update) restricted as in Eq. (Cupdate); ``abp_grid_apply_hills``,
   no atomics), so replicas that start equal stay bit-identical and equal one
   grid that received all walkers' hills;
4. ``forces``: the look-up of V_b and its gradient and the chain rule
   (Eq. (btraj-grad); ``abp_shared_forces``).

Only the hill records cross ranks (48 bytes per hill), never coordinates,
forces or grid nodes: the paper's rule of moving only what the bias needs
(SI, Minimization of Interprocess Communications), applied to the bias
itself. ``shared_step`` runs steps 1-4 against any replica object with
``hills``/``apply``/``forces`` methods; ``GpuReplica`` is the one backed by
the CUDA library.
"""
from __future__ import annotations

import numpy as np

from . import abp

HILL_DTYPE = abp.HILL_DTYPE


def gather_hills(local: np.ndarray, group=None) -> np.ndarray:
    """All-gather hill records (HILL_DTYPE) over torch.distributed, in rank
    order. Without an initialised process group (or with one rank) the local
    records are returned. The records travel as raw bytes: every rank
    receives them bit for bit."""
    local = np.ascontiguousarray(local, dtype=HILL_DTYPE)
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return local.copy()
    world = dist.get_world_size(group)
    if world == 1:
        return local.copy()
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    n = torch.tensor([local.shape[0]], dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    if m == 0:
        return np.zeros(0, dtype=HILL_DTYPE)
    item = HILL_DTYPE.itemsize
    buf = np.zeros(m * item, dtype=np.uint8)
    buf[: local.nbytes] = local.view(np.uint8)
    mine = torch.from_numpy(buf).to(dev)
    parts = [torch.empty(m * item, dtype=torch.uint8, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    out = [p.cpu().numpy()[: c * item].view(HILL_DTYPE) for p, c in zip(parts, counts)]
    return np.concatenate(out).copy()


def shared_step(replica, coords, coord_offsets, forces, force_offsets, step: int,
                mode: int = abp.ABP_FORCES_OVERWRITE, group=None, exchange=gather_hills) -> np.ndarray:
    """One MD step of this rank's walkers on a replicated shared grid.
    Returns the step's hill records of all ranks, in the order applied."""
    local = replica.hills(coords, coord_offsets, step)
    every = exchange(local, group)
    if every.shape[0]:
        replica.apply(every)
    replica.forces(forces, force_offsets, mode, step)
    return every


class GpuReplica:
    """This rank's walkers (``abp.Walker`` objects of one context, all on one
    grid created with shared = 1) and that grid: the rank's replica."""

    def __init__(self, ctx, walkers, dtype: int = abp.ABP_F32):
        if not walkers:
            raise ValueError("a replica needs at least one walker")
        grids = {w.grid for w in walkers}
        if len(grids) != 1:
            raise ValueError("the walkers of a replica share one grid")
        self.ctx, self.walkers, self.dtype = ctx, list(walkers), dtype

    def hills(self, coords, coord_offsets, step: int) -> np.ndarray:
        return abp.abp_shared_hills(self.ctx.handle, self.walkers, coords, self.dtype, coord_offsets, step)

    def apply(self, hills: np.ndarray):
        abp.abp_grid_apply_hills(self.ctx.handle, self.walkers[0], hills)

    def forces(self, forces, force_offsets, mode: int, step: int):
        abp.abp_shared_forces(self.ctx.handle, self.walkers, forces, self.dtype, force_offsets, mode, step)
