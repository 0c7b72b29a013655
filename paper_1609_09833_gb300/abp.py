"""Python binding of the C ABI in include/abp.h (argument marshalling only).

Every function named ``abp_*`` here calls the C entry point of the same name
in the in-tree CUDA library ``_build/libabp.so``; every step of the force call
runs in that library's kernels. PyTorch supplies device memory and streams.
There is no CPU fallback: if the library is missing or fails to load, the
import of this module's functions raises.

Higher-level helpers (``Context``) turn the plain-data walker specs of
``paper_1609_09833_gb300.synth`` into descriptors and keep handles alive.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ABP_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "ADMISSION", -5: "NONFINITE", -6: "TIMEOUT",
          -7: "UNSUPPORTED"}
ABP_ERR_INVALID_ARG, ABP_ERR_CUDA, ABP_ERR_OOM, ABP_ERR_ADMISSION = -1, -2, -3, -4
ABP_ERR_NONFINITE, ABP_ERR_TIMEOUT, ABP_ERR_UNSUPPORTED, ABP_ERR_CANCELLED = -5, -6, -7, -8
CV_TYPES = {"com_dist": 0, "dihedral": 1, "coord": 2, "rmsd": 3}
ABP_METHOD_WT, ABP_METHOD_MABP = 0, 1
ABP_PREC_FP32_COMP, ABP_PREC_FP64 = 0, 1
ABP_F32, ABP_F64 = 0, 1
ABP_FORCES_ACCUMULATE, ABP_FORCES_OVERWRITE = 0, 1
WFLAG_DEPOSIT, WFLAG_OOR, WFLAG_SINGULAR, WFLAG_NONFINITE = 1, 2, 4, 8


class AbpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ABP_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("ncv", C.c_int), ("n", C.c_int * 3), ("periodic", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("precision", C.c_int), ("shared", C.c_int)]


class CvDesc(C.Structure):
    _fields_ = [("type", C.c_int), ("n_a", C.c_int), ("n_b", C.c_int), ("idx_a", C.POINTER(C.c_int32)),
                ("idx_b", C.POINTER(C.c_int32)), ("mass_a", C.POINTER(C.c_double)),
                ("mass_b", C.POINTER(C.c_double)), ("r0", C.c_double), ("nn", C.c_int), ("mm", C.c_int),
                ("pbc", C.c_int), ("box", C.c_double * 3), ("ref", C.POINTER(C.c_double))]


class WalkerDesc(C.Structure):
    _fields_ = [("natoms", C.c_int), ("cv", CvDesc * 3), ("w", C.c_double), ("sigma", C.c_double * 3),
                ("cutoff", C.c_double), ("gamma", C.c_double), ("kT", C.c_double), ("stride", C.c_int64),
                ("method", C.c_int), ("a", C.c_double * 3), ("p", C.c_int), ("b", C.c_double), ("c", C.c_double),
                ("smax", C.c_double * 3), ("kwall", C.c_double)]


class DepositRec(C.Structure):
    _fields_ = [("step", C.c_int64), ("walker_id", C.c_int32), ("ic", C.c_int32 * 3), ("s", C.c_double * 3),
                ("height", C.c_double)]


# abp_hill: one hill record of a shared-grid exchange (48 bytes)
HILL_DTYPE = np.dtype([("s", "<f8", (3,)), ("height", "<f8"), ("step", "<i8"), ("walker_id", "<i4"),
                       ("pad", "<i4")])
assert HILL_DTYPE.itemsize == 48


class MdDesc(C.Structure):
    _fields_ = [("dt", C.c_double), ("mobility", C.c_double), ("kT", C.c_double), ("seed", C.c_uint64),
                ("potential", C.c_int), ("dw_a", C.c_double), ("dw_b", C.c_double), ("mb_scale", C.c_double),
                ("mb_map", C.c_double * 4), ("mb_A", C.c_double * 4), ("mb_a", C.c_double * 4),
                ("mb_b", C.c_double * 4), ("mb_c", C.c_double * 4), ("mb_x0", C.c_double * 4),
                ("mb_y0", C.c_double * 4)]


ABP_POT_NONE, ABP_POT_DOUBLE_WELL, ABP_POT_MULLER_BROWN = 0, 1, 2
_POTS = {"none": ABP_POT_NONE, "double_well": ABP_POT_DOUBLE_WELL, "muller_brown": ABP_POT_MULLER_BROWN}


def md_desc(md: dict) -> MdDesc:
    """MdDesc from a closed-loop dynamics dict (synth.md_params)."""
    d = MdDesc()
    d.dt, d.mobility, d.kT = float(md["dt"]), float(md["mu"]), float(md["kT"])
    d.seed = int(md["seed"]) & ((1 << 64) - 1)
    d.potential = _POTS[md.get("potential", "none")]
    if d.potential == ABP_POT_DOUBLE_WELL:
        d.dw_a, d.dw_b = float(md["dw"][0]), float(md["dw"][1])
    elif d.potential == ABP_POT_MULLER_BROWN:
        mb = md["mb"]
        d.mb_scale = float(mb["scale"])
        for q in range(4):
            d.mb_map[q] = float(mb["map"][q])
            for key in ("A", "a", "b", "c", "x0", "y0"):
                getattr(d, "mb_" + key)[q] = float(mb[key][q])
    return d


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double)]


ABP_TUNE_TIMING = 5


class ServerDesc(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("max_atoms", C.c_int), ("nstreams", C.c_int)]


class Result(C.Structure):
    _fields_ = [("sim", C.c_int64), ("step", C.c_int64), ("tag", C.c_uint64), ("t_submit", C.c_double),
                ("t_done", C.c_double), ("status", C.c_int32), ("batch", C.c_int32)]


_vp, _i64p = C.c_void_p, C.POINTER(C.c_int64)
_SIGS = {
    "abp_ctx_create": [C.POINTER(_vp), C.c_int, _vp, C.c_size_t],
    "abp_ctx_set_stream": [_vp, _vp],
    "abp_ctx_bytes": [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
    "abp_ctx_tune": [_vp, C.c_int, C.c_int],
    "abp_ctx_destroy": [_vp],
    "abp_create_grid": [_vp, C.POINTER(GridDesc), C.POINTER(_vp)],
    "abp_grid_destroy": [_vp],
    "abp_grid_clear": [_vp, _vp],
    "abp_walker_create": [_vp, _vp, C.POINTER(WalkerDesc), C.POINTER(_vp)],
    "abp_walker_destroy": [_vp],
    "abp_walker_id": [_vp],
    "abp_step": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, C.c_int64],
    "abp_forces": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, C.c_int],
    "abp_run": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, C.c_int64, _vp, _vp, C.c_int64, C.c_int,
                C.c_int64, C.c_int],
    "abp_step_plain": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, _vp, _vp, C.c_int, C.c_int64],
    "abp_md_run": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, C.POINTER(MdDesc), C.POINTER(C.c_uint32), _vp,
                   _vp, C.c_int64, _vp, _vp, C.c_int64, C.c_int, C.c_int64, C.c_int],
    "abp_shared_hills": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, C.c_int64, _vp, C.c_size_t,
                         C.POINTER(C.c_size_t)],
    "abp_grid_apply_hills": [_vp, _vp, _vp, C.c_size_t],
    "abp_shared_forces": [_vp, C.POINTER(_vp), C.c_int, _vp, C.c_int, _vp, C.c_int, C.c_int64],
    "abp_grid_record_bytes": [_vp],
    "abp_grid_save": [_vp, _vp, _vp, C.c_int],
    "abp_grid_restore": [_vp, _vp, _vp, C.c_int],
    "abp_bias_readout": [_vp, _vp, _vp, C.c_int, C.c_int],
    "abp_bias_upload": [_vp, _vp, _vp, C.c_int, C.c_int],
    "abp_walker_readout": [_vp, _vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                           C.POINTER(C.c_int)],
    "abp_deposit_log_enable": [_vp, C.c_size_t],
    "abp_deposit_log_readout": [_vp, C.POINTER(DepositRec), C.c_size_t, C.POINTER(C.c_size_t),
                                C.POINTER(C.c_size_t)],
    "abp_deposit_log_clear": [_vp],
    "abp_sync": [_vp],
    "abp_step_static": [C.c_int, _vp, C.POINTER(GridDesc), _vp, C.POINTER(WalkerDesc), _vp, C.c_int, _vp, C.c_int,
                        C.c_int64],
    "abp_server_create": [_vp, C.POINTER(ServerDesc), C.POINTER(_vp)],
    "abp_server_destroy": [_vp],
    "abp_server_admit": [_vp, C.POINTER(GridDesc), C.POINTER(WalkerDesc), C.POINTER(C.c_int64)],
    "abp_server_release": [_vp, C.c_int64],
    "abp_server_bias_readout": [_vp, C.c_int64, _vp, C.c_int, C.c_int],
    "abp_server_submit": [_vp, C.c_int64, C.c_int64, _vp, _vp, C.c_uint64],
    "abp_server_submit_many": [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp],
    "abp_server_cancel": [_vp, C.c_int64, C.POINTER(C.c_int64)],
    "abp_server_poll": [_vp, C.POINTER(Result), C.c_int, C.POINTER(C.c_int), C.c_int],
    "abp_server_stats": [_vp, _i64p, _i64p, _i64p, _i64p],
    "abp_server_times": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                         C.POINTER(C.c_double)],
    "abp_server_now": [],
    "abp_checked_violations": [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_int)],
    "abp_fp32_fma_peak": [C.c_int, _vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "abp_kernel_times": [_vp, C.POINTER(KernelTime), C.c_int, C.POINTER(C.c_int)],
    "abp_last_error": [],
    "abp_version": [],
}
_VOID = {"abp_ctx_destroy", "abp_grid_destroy", "abp_walker_destroy", "abp_server_destroy"}
_STR = {"abp_last_error", "abp_version"}

_lib_handle = None


def lib_path() -> str:
    """The in-tree library; ABP_LIBRARY names another build of it (the
    checked build, for instance)."""
    return os.environ.get("ABP_LIBRARY") or _build.LIB


def load():
    """Load the CUDA library (raises if it is not built)."""
    global _lib_handle
    if _lib_handle is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing (run paper_1609_09833_gb300.build)")
        L = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in _VOID else (C.c_char_p if name in _STR else C.c_int)
        L.abp_walker_id.restype = C.c_int32
        L.abp_grid_record_bytes.restype = C.c_size_t
        L.abp_server_now.restype = C.c_double
        _lib_handle = L
    return _lib_handle


def exported_symbols():
    return list(_SIGS)


def _check(rc: int):
    if rc != ABP_OK:
        raise AbpError(rc, load().abp_last_error().decode())
    return rc


def _ptr(t) -> int:
    """Device (or host) address of a torch tensor / numpy array / int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def walker_array(ws):
    """The C array of walker handles a call takes; a caller that calls every
    MD step can build it once and pass it in place of the list."""
    return (_vp * max(1, len(ws)))(*[w.handle if hasattr(w, "handle") else w for w in ws])


def _walkers(ws):
    return ws if isinstance(ws, C.Array) else walker_array(ws)


# ---------------------------------------------------------------- raw ABI names


def abp_ctx_create(device: int = 0, stream=None, budget: int = 0):
    h = _vp()
    _check(load().abp_ctx_create(C.byref(h), int(device), stream, int(budget)))
    return h.value


def abp_ctx_set_stream(ctx, stream):
    _check(load().abp_ctx_set_stream(ctx, stream))


def abp_ctx_bytes(ctx):
    u, b = C.c_size_t(), C.c_size_t()
    _check(load().abp_ctx_bytes(ctx, C.byref(u), C.byref(b)))
    return u.value, b.value


ABP_TUNE_GROUP_THREADS, ABP_TUNE_GROUPS_PER_CTA, ABP_TUNE_TILE, ABP_TUNE_LEAN = 1, 2, 3, 4


def abp_ctx_tune(ctx, knob: int, value: int):
    _check(load().abp_ctx_tune(ctx, int(knob), int(value)))


def abp_ctx_destroy(ctx):
    load().abp_ctx_destroy(ctx)


def abp_create_grid(ctx, desc: GridDesc):
    h = _vp()
    _check(load().abp_create_grid(ctx, C.byref(desc), C.byref(h)))
    return h.value


def abp_grid_destroy(g):
    load().abp_grid_destroy(g)


def abp_grid_clear(ctx, g):
    _check(load().abp_grid_clear(ctx, g))


def abp_walker_create(ctx, grid, desc: WalkerDesc):
    h = _vp()
    _check(load().abp_walker_create(ctx, grid, C.byref(desc), C.byref(h)))
    return h.value


def abp_walker_destroy(w):
    load().abp_walker_destroy(w)


def abp_walker_id(w) -> int:
    return int(load().abp_walker_id(w))


def abp_step(ctx, walkers, coords, coords_dtype, coord_offsets, step: int):
    _check(load().abp_step(ctx, _walkers(walkers), len(walkers), _ptr(coords), coords_dtype, _ptr(coord_offsets),
                           int(step)))


def abp_forces(ctx, walkers, forces, forces_dtype, force_offsets, mode=ABP_FORCES_ACCUMULATE):
    _check(load().abp_forces(ctx, _walkers(walkers), len(walkers), _ptr(forces), forces_dtype, _ptr(force_offsets),
                             int(mode)))


def abp_run(ctx, walkers, coords, coords_dtype, coord_offsets, coord_step_stride, forces, force_offsets,
            force_step_stride, mode, step0, nsteps):
    _check(load().abp_run(ctx, _walkers(walkers), len(walkers), _ptr(coords), coords_dtype, _ptr(coord_offsets),
                          int(coord_step_stride), _ptr(forces), _ptr(force_offsets), int(force_step_stride),
                          int(mode), int(step0), int(nsteps)))


def abp_step_plain(ctx, walkers, coords, coords_dtype, coord_offsets, forces, force_offsets, mode, step):
    _check(load().abp_step_plain(ctx, _walkers(walkers), len(walkers), _ptr(coords), coords_dtype,
                                 _ptr(coord_offsets), _ptr(forces), _ptr(force_offsets), int(mode), int(step)))


def abp_md_run(ctx, walkers, coords, coords_dtype, coord_offsets, md, streams, traj=None, traj_offsets=None,
               traj_step_stride=0, forces=None, force_offsets=None, force_step_stride=0, mode=ABP_FORCES_OVERWRITE,
               step0: int = 0, nsteps: int = 1):
    """Closed-loop MD steps (coordinates moved in place). md: MdDesc or a
    dynamics dict; streams: one noise stream per walker."""
    desc = md if isinstance(md, MdDesc) else md_desc(md)
    st = streams if (isinstance(streams, np.ndarray) and streams.dtype == np.uint32 and streams.flags.c_contiguous) \
        else np.ascontiguousarray(np.asarray(streams, dtype=np.uint32))
    _check(load().abp_md_run(ctx, _walkers(walkers), len(walkers), _ptr(coords), coords_dtype, _ptr(coord_offsets),
                             C.byref(desc), st.ctypes.data_as(C.POINTER(C.c_uint32)), _ptr(traj), _ptr(traj_offsets),
                             int(traj_step_stride), _ptr(forces), _ptr(force_offsets), int(force_step_stride),
                             int(mode), int(step0), int(nsteps)))


def abp_shared_hills(ctx, walkers, coords, coords_dtype, coord_offsets, step: int) -> np.ndarray:
    """Hill records (HILL_DTYPE) of this step's depositing walkers, in list order."""
    out = np.zeros(max(1, len(walkers)), dtype=HILL_DTYPE)
    n = C.c_size_t()
    _check(load().abp_shared_hills(ctx, _walkers(walkers), len(walkers), _ptr(coords), coords_dtype,
                                   _ptr(coord_offsets), int(step), out.ctypes.data, out.shape[0], C.byref(n)))
    return out[:n.value].copy()


def abp_grid_apply_hills(ctx, shape_walker, hills: np.ndarray):
    h = np.ascontiguousarray(hills, dtype=HILL_DTYPE)
    w = shape_walker.handle if hasattr(shape_walker, "handle") else shape_walker
    _check(load().abp_grid_apply_hills(ctx, w, h.ctypes.data if h.shape[0] else None, h.shape[0]))


def abp_shared_forces(ctx, walkers, forces, forces_dtype, force_offsets, mode, step: int):
    _check(load().abp_shared_forces(ctx, _walkers(walkers), len(walkers), _ptr(forces), forces_dtype,
                                    _ptr(force_offsets), int(mode), int(step)))


def abp_grid_record_bytes(grid) -> int:
    return int(load().abp_grid_record_bytes(grid))


def abp_grid_save(ctx, grid) -> np.ndarray:
    """The grid's raw node records (and shadow) as host bytes."""
    out = np.zeros(abp_grid_record_bytes(grid), dtype=np.uint8)
    _check(load().abp_grid_save(ctx, grid, out.ctypes.data, 0))
    return out


def abp_grid_restore(ctx, grid, data: np.ndarray):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    if data.nbytes != abp_grid_record_bytes(grid):
        raise ValueError("record bytes do not match the grid")
    _check(load().abp_grid_restore(ctx, grid, data.ctypes.data, 0))


def abp_bias_readout(ctx, grid, dst, dst_is_device: bool, dtype: int):
    _check(load().abp_bias_readout(ctx, grid, _ptr(dst), int(dst_is_device), int(dtype)))


def abp_bias_upload(ctx, grid, src, src_is_device: bool, dtype: int):
    _check(load().abp_bias_upload(ctx, grid, _ptr(src), int(src_is_device), int(dtype)))


def abp_walker_readout(ctx, w):
    s, dV = (C.c_double * 3)(), (C.c_double * 3)()
    V, fl = C.c_double(), C.c_int()
    rc = load().abp_walker_readout(ctx, w, s, C.byref(V), dV, C.byref(fl))
    out = {"s": np.array(list(s)), "V": V.value, "dV": np.array(list(dV)), "flags": fl.value}
    if rc not in (ABP_OK, ABP_ERR_NONFINITE):
        _check(rc)
    out["status"] = rc
    return out


def abp_deposit_log_enable(ctx, capacity: int):
    _check(load().abp_deposit_log_enable(ctx, int(capacity)))


def abp_deposit_log_readout(ctx, cap: int):
    buf = (DepositRec * max(1, cap))()
    n, tot = C.c_size_t(), C.c_size_t()
    _check(load().abp_deposit_log_readout(ctx, buf, int(cap), C.byref(n), C.byref(tot)))
    k = n.value
    return {
        "step": np.array([buf[i].step for i in range(k)], dtype=np.int64),
        "walker_id": np.array([buf[i].walker_id for i in range(k)], dtype=np.int32),
        "ic": np.array([list(buf[i].ic) for i in range(k)], dtype=np.int32).reshape(k, 3),
        "s": np.array([list(buf[i].s) for i in range(k)]).reshape(k, 3),
        "height": np.array([buf[i].height for i in range(k)]),
        "total": tot.value,
    }


def abp_deposit_log_clear(ctx):
    _check(load().abp_deposit_log_clear(ctx))


def abp_sync(ctx):
    _check(load().abp_sync(ctx))


def abp_step_static(device, stream, grid_desc: GridDesc, grid_records, walker_desc: WalkerDesc, coords,
                    coords_dtype, forces, mode, step):
    _check(load().abp_step_static(int(device), stream, C.byref(grid_desc), _ptr(grid_records), C.byref(walker_desc),
                                  _ptr(coords), int(coords_dtype), _ptr(forces), int(mode), int(step)))


def abp_server_create(ctx, max_batch=0, max_atoms=0, nstreams=0):
    d = ServerDesc(int(max_batch), int(max_atoms), int(nstreams))
    h = _vp()
    _check(load().abp_server_create(ctx, C.byref(d), C.byref(h)))
    return h.value


def abp_server_destroy(srv):
    load().abp_server_destroy(srv)


def abp_server_admit(srv, grid: GridDesc, walker: WalkerDesc) -> int:
    sim = C.c_int64()
    _check(load().abp_server_admit(srv, C.byref(grid), C.byref(walker), C.byref(sim)))
    return sim.value


def abp_server_release(srv, sim: int):
    _check(load().abp_server_release(srv, int(sim)))


def abp_server_bias_readout(srv, sim: int, spec_grid: dict) -> np.ndarray:
    """A served simulation's grid fields [nodes, 1 + d] (FP64), after its requests."""
    d = len(spec_grid["n"])
    out = np.zeros((int(np.prod(spec_grid["n"])), 1 + d), dtype=np.float64)
    _check(load().abp_server_bias_readout(srv, int(sim), _ptr(out), 0, ABP_F64))
    return out


def abp_server_submit(srv, sim: int, step: int, coords_host, forces_host, tag: int = 0):
    _check(load().abp_server_submit(srv, int(sim), int(step), _ptr(coords_host), _ptr(forces_host), int(tag)))


def abp_server_submit_many(srv, sims, steps, coords_host, forces_host, tags=None):
    sims = np.ascontiguousarray(sims, dtype=np.int64)
    steps = np.ascontiguousarray(steps, dtype=np.int64)
    tg = None if tags is None else np.ascontiguousarray(tags, dtype=np.uint64)
    _check(load().abp_server_submit_many(srv, len(sims), _ptr(sims), _ptr(steps), _ptr(coords_host),
                                         _ptr(forces_host), _ptr(tg)))


def abp_server_cancel(srv, sim) -> int:
    n = C.c_int64()
    _check(load().abp_server_cancel(srv, int(sim), C.byref(n)))
    return int(n.value)


def abp_server_poll(srv, cap: int = 4096, wait_ms: int = 0):
    buf = (Result * max(1, cap))()
    n = C.c_int()
    _check(load().abp_server_poll(srv, buf, int(cap), C.byref(n), int(wait_ms)))
    return [buf[i] for i in range(n.value)]


def abp_server_stats(srv):
    v = [C.c_int64() for _ in range(4)]
    _check(load().abp_server_stats(srv, *[C.byref(x) for x in v]))
    return {"submitted": v[0].value, "finished": v[1].value, "launches": v[2].value, "queued": v[3].value}


def abp_server_times(srv):
    v = [C.c_double() for _ in range(4)]
    _check(load().abp_server_times(srv, *[C.byref(x) for x in v]))
    return {"fill": v[0].value, "launch": v[1].value, "complete": v[2].value, "wait": v[3].value}


def abp_checked_violations(ctx):
    """(out-of-grid node indices counted, whether the library is the checked build)."""
    n, chk = C.c_uint64(), C.c_int()
    _check(load().abp_checked_violations(ctx, C.byref(n), C.byref(chk)))
    return int(n.value), bool(chk.value)


def abp_server_now() -> float:
    return float(load().abp_server_now())


def abp_kernel_times(ctx) -> dict:
    """Per-kernel {name: (launches, ms)} since the last call (ABP_TUNE_TIMING on)."""
    buf = (KernelTime * 64)()
    n = C.c_int()
    _check(load().abp_kernel_times(ctx, buf, 64, C.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(n.value)}


def abp_fp32_fma_peak(device: int = 0, stream=None, iters: int = 20000):
    """Measured FP32 FMA throughput of the device: (FLOP/s, seconds timed)."""
    f, s = C.c_double(), C.c_double()
    _check(load().abp_fp32_fma_peak(int(device), stream, int(iters), C.byref(f), C.byref(s)))
    return f.value, s.value


def abp_last_error() -> str:
    return load().abp_last_error().decode()


def abp_version() -> str:
    return load().abp_version().decode()


# ---------------------------------------------------------------- spec marshalling


def grid_desc(spec_grid: dict, precision: int = ABP_PREC_FP32_COMP, shared: bool = False) -> GridDesc:
    d = GridDesc()
    n = spec_grid["n"]
    d.ncv = len(n)
    for k in range(len(n)):
        d.n[k] = int(n[k])
        d.periodic[k] = int(bool(spec_grid["periodic"][k]))
        d.lo[k] = float(spec_grid["lo"][k])
        d.hi[k] = float(spec_grid["hi"][k])
    d.precision = int(precision)
    d.shared = int(bool(shared))
    return d


def walker_desc(spec: dict):
    """WalkerDesc for a walker spec, plus the arrays it points at (keep alive)."""
    d = WalkerDesc()
    keep = []
    d.natoms = int(spec["natoms"])
    for k, cv in enumerate(spec["cvs"]):
        c = d.cv[k]
        c.type = CV_TYPES[cv["type"]]
        a = np.ascontiguousarray(cv["a"], dtype=np.int32)
        b = np.ascontiguousarray(cv.get("b", np.zeros(0)), dtype=np.int32)
        keep += [a, b]
        c.n_a, c.n_b = len(a), len(b)
        c.idx_a = a.ctypes.data_as(C.POINTER(C.c_int32))
        c.idx_b = b.ctypes.data_as(C.POINTER(C.c_int32)) if len(b) else None
        for key in ("ma", "mb"):
            m = cv.get(key)
            if m is not None:
                m = np.ascontiguousarray(m, dtype=np.float64)
                keep.append(m)
                setattr(c, "mass_a" if key == "ma" else "mass_b", m.ctypes.data_as(C.POINTER(C.c_double)))
        c.r0 = float(cv.get("r0", 0.4))
        c.nn = int(cv.get("n", 6))
        c.mm = int(cv.get("m", 12))
        c.pbc = int(bool(cv.get("pbc", False)))
        box = cv.get("box", (0.0, 0.0, 0.0))
        for q in range(3):
            c.box[q] = float(box[q])
        if cv["type"] == "rmsd":
            ref = np.ascontiguousarray(cv["ref"], dtype=np.float64).reshape(-1)
            keep.append(ref)
            c.ref = ref.ctypes.data_as(C.POINTER(C.c_double))
    hl = spec["hill"]
    d.w = float(hl["w"])
    d.kT = float(hl["kT"])
    d.stride = int(hl["stride"])
    if hl.get("kwall", 0.0) > 0:
        d.kwall = float(hl["kwall"])
        for k, v in enumerate(hl["smax"]):
            d.smax[k] = float(v)
    if hl.get("method", "wt") == "mabp":
        d.method = ABP_METHOD_MABP
        for k, a in enumerate(hl["a"]):
            d.a[k] = float(a)
        d.p = int(hl["p"])
        d.b = float(hl["b"])
        d.c = float(hl["c"])
    else:
        for k, s in enumerate(hl["sigma"]):
            d.sigma[k] = float(s)
        d.cutoff = float(hl["cutoff"])
        d.gamma = float(hl["gamma"])
    return d, keep


class Walker:
    def __init__(self, ctx: "Context", handle: int, grid: int, spec: dict):
        self.ctx, self.handle, self.grid, self.spec = ctx, handle, grid, spec
        self.id = abp_walker_id(handle)
        self.d = len(spec["grid"]["n"])
        self.nodes = int(np.prod(spec["grid"]["n"]))


class Context:
    """Owns an abp_ctx and the grids/walkers made from specs."""

    def __init__(self, device: int = 0, stream=None, budget: int = 0):
        import torch

        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self.handle = abp_ctx_create(device, stream, budget)
        self.grids = []
        self.walkers = []

    def set_stream(self, stream):
        abp_ctx_set_stream(self.handle, stream)

    def make_grid(self, spec_grid: dict, precision: int = ABP_PREC_FP32_COMP, shared: bool = False) -> int:
        g = abp_create_grid(self.handle, grid_desc(spec_grid, precision, shared))
        self.grids.append(g)
        return g

    def make_walkers(self, specs, precision: int = ABP_PREC_FP32_COMP):
        """One walker per spec; specs with the same "shared" key share one grid."""
        out, shared = [], {}
        for sp in specs:
            key = sp.get("shared")
            if key is not None and key in shared:
                g = shared[key]
            else:
                g = self.make_grid(sp["grid"], precision, shared=key is not None)
                if key is not None:
                    shared[key] = g
            desc, keep = walker_desc(sp)
            h = abp_walker_create(self.handle, g, desc)
            del keep
            w = Walker(self, h, g, sp)
            self.walkers.append(w)
            out.append(w)
        return out

    def bias(self, walker_or_grid, dtype=ABP_F64) -> np.ndarray:
        g = walker_or_grid.grid if isinstance(walker_or_grid, Walker) else walker_or_grid
        spec = walker_or_grid.spec if isinstance(walker_or_grid, Walker) else None
        d = walker_or_grid.d if spec else None
        if d is None:
            raise ValueError("pass a Walker")
        out = np.zeros((walker_or_grid.nodes, 1 + d), dtype=np.float64 if dtype == ABP_F64 else np.float32)
        abp_bias_readout(self.handle, g, out, False, dtype)
        return out

    def upload_bias(self, walker: Walker, field: np.ndarray):
        field = np.ascontiguousarray(field, dtype=np.float64)
        assert field.shape == (walker.nodes, 1 + walker.d)
        abp_bias_upload(self.handle, walker.grid, field, False, ABP_F64)

    def readout(self, walker: Walker):
        return abp_walker_readout(self.handle, walker.handle)

    def close(self):
        for w in self.walkers:
            abp_walker_destroy(w.handle)
        for g in self.grids:
            abp_grid_destroy(g)
        self.walkers, self.grids = [], []
        if self.handle:
            abp_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_records(frames, dtype=None):
    """[T, atoms, 3] array -> contiguous [T, atoms, 4] records (pad 0) as a torch tensor on the GPU."""
    import torch

    t = torch.as_tensor(np.ascontiguousarray(frames))
    if dtype is not None:
        t = t.to(dtype)
    rec = torch.zeros(t.shape[:-1] + (4,), dtype=t.dtype)
    rec[..., :3] = t
    return rec
