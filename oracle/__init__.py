"""FP64 CPU oracle for the adaptive-biasing-potential force call.

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library
never calls it and shares no code with it; the only things both sides consume
are the plain-data walker specs and frames made by the seeded input
generators.

The arithmetic lives in ``abp_oracle.c`` (plain C, double precision, one
function per step of the method, each citing the paper's equation). This
module compiles it with gcc, mirrors its structs with ctypes and converts
walker specs (dicts, see ``paper_1609_09833_gb300.synth``) into them.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, finite differences, exactness on multilinear fields, brute
force on tiny grids, rational arithmetic for the switching function and
well-tempered convergence on an analytic double well).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CV_TYPES = {"com_dist": 0, "dihedral": 1, "coord": 2, "pos_x": 3, "rmsd": 4}
METHODS = {"wt": 0, "mabp": 1}
FLAG_DEPOSIT, FLAG_OOR, FLAG_SINGULAR, FLAG_BADARG = 1, 2, 4, 8
MAXCV = 3


class OrCv(C.Structure):
    _fields_ = [
        ("type", C.c_int),
        ("na", C.c_int),
        ("nb", C.c_int),
        ("ia", C.POINTER(C.c_int)),
        ("ib", C.POINTER(C.c_int)),
        ("ma", C.POINTER(C.c_double)),
        ("mb", C.POINTER(C.c_double)),
        ("r0", C.c_double),
        ("nn", C.c_int),
        ("mm", C.c_int),
        ("pbc", C.c_int),
        ("box", C.c_double * 3),
        ("ref", C.POINTER(C.c_double)),
    ]


class OrGrid(C.Structure):
    _fields_ = [
        ("d", C.c_int),
        ("n", C.c_int * 3),
        ("periodic", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
    ]


class OrHill(C.Structure):
    _fields_ = [
        ("w", C.c_double),
        ("sigma", C.c_double * 3),
        ("cutoff", C.c_double),
        ("gamma", C.c_double),
        ("kT", C.c_double),
        ("stride", C.c_int64),
        ("method", C.c_int),
        ("a", C.c_double * 3),
        ("p", C.c_int),
        ("b", C.c_double),
        ("c", C.c_double),
        ("smax", C.c_double * 3),
        ("kwall", C.c_double),
    ]


class OrWalker(C.Structure):
    _fields_ = [("g", OrGrid), ("hill", OrHill), ("cv", OrCv * MAXCV), ("natoms", C.c_int)]


class OrMd(C.Structure):
    _fields_ = [
        ("dt", C.c_double),
        ("mu", C.c_double),
        ("kT", C.c_double),
        ("seed", C.c_uint64),
        ("pot", C.c_int),
        ("dw_a", C.c_double),
        ("dw_b", C.c_double),
        ("mb_scale", C.c_double),
        ("mb_map", C.c_double * 4),
        ("mb_A", C.c_double * 4),
        ("mb_a", C.c_double * 4),
        ("mb_b", C.c_double * 4),
        ("mb_c", C.c_double * 4),
        ("mb_x0", C.c_double * 4),
        ("mb_y0", C.c_double * 4),
        ("state_f32", C.c_int),
    ]


POTENTIALS = {"none": 0, "double_well": 1, "muller_brown": 2}


def md_struct(md: dict) -> OrMd:
    """An or_md from a closed-loop dynamics dict (see synth.md_params)."""
    m = OrMd()
    m.dt, m.mu, m.kT = float(md["dt"]), float(md["mu"]), float(md["kT"])
    m.seed = int(md["seed"]) & ((1 << 64) - 1)
    m.pot = POTENTIALS[md.get("potential", "none")]
    m.state_f32 = int(bool(md.get("state_f32", False)))
    if m.pot == POTENTIALS["double_well"]:
        m.dw_a, m.dw_b = float(md["dw"][0]), float(md["dw"][1])
    elif m.pot == POTENTIALS["muller_brown"]:
        mb = md["mb"]
        m.mb_scale = float(mb["scale"])
        for q in range(4):
            m.mb_map[q] = float(mb["map"][q])
            for key in ("A", "a", "b", "c", "x0", "y0"):
                getattr(m, "mb_" + key)[q] = float(mb[key][q])
    return m


class OrStepAux(C.Structure):
    _fields_ = [("H", C.c_double * 9), ("A", C.c_double * 4), ("sb", C.c_double * 3)]


class OrDeposit(C.Structure):
    _fields_ = [
        ("step", C.c_int64),
        ("walker", C.c_int32),
        ("ic", C.c_int32 * 3),
        ("s", C.c_double * 3),
        ("height", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile abp_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.or_cv_eval.argtypes = [C.POINTER(OrCv), C.c_int, dp, dp, dp]
        L.or_cv_eval.restype = C.c_int
        L.or_switch.argtypes = [C.c_double, C.c_int, C.c_int, dp]
        L.or_switch.restype = C.c_double
        L.or_interp.argtypes = [C.POINTER(OrGrid), dp, dp, dp, dp]
        L.or_interp.restype = C.c_int
        L.or_height.argtypes = [C.POINTER(OrHill), C.c_double]
        L.or_height.restype = C.c_double
        L.or_deposit_hill.argtypes = [C.POINTER(OrGrid), C.POINTER(OrHill), dp, dp, C.c_double, ip, dp]
        L.or_deposit_hill.restype = None
        L.or_grid_nodes.argtypes = [C.POINTER(OrGrid)]
        L.or_grid_nodes.restype = C.c_long
        L.or_stencil_halfwidth.argtypes = [C.POINTER(OrGrid), C.POINTER(OrHill), C.c_int]
        L.or_stencil_halfwidth.restype = C.c_int
        L.or_check.argtypes = [C.POINTER(OrGrid), C.POINTER(OrHill)]
        L.or_check.restype = C.c_int
        L.or_batch_step.argtypes = [
            C.c_int, C.POINTER(OrWalker), C.POINTER(dp), C.POINTER(dp), C.c_int64,
            dp, dp, dp, C.POINTER(dp), ip, C.POINTER(OrDeposit), C.POINTER(OrMd), C.POINTER(C.c_uint32),
            C.POINTER(dp), C.POINTER(OrStepAux), C.POINTER(dp), C.POINTER(dp),
        ]
        L.or_batch_step.restype = C.c_int
        u32p = C.POINTER(C.c_uint32)
        L.or_run.argtypes = [
            C.c_int, C.POINTER(OrWalker), C.POINTER(dp), dp, C.POINTER(C.c_int64), C.c_int64,
            C.c_int64, C.c_int64, dp, dp, dp, dp, ip, C.POINTER(OrDeposit), C.c_int64,
            C.POINTER(C.c_int64), C.POINTER(OrMd), u32p, dp, C.POINTER(OrStepAux), dp, C.POINTER(dp),
        ]
        L.or_interp_aux.argtypes = [C.POINTER(OrGrid), dp, dp, dp, dp, dp]
        L.or_interp_aux.restype = None
        L.or_cv_round_bound.argtypes = [C.POINTER(OrCv), dp]
        L.or_cv_round_bound.restype = C.c_double
        L.or_md_run.argtypes = [
            C.c_int, C.POINTER(OrWalker), C.POINTER(dp), dp, C.POINTER(C.c_int64), C.c_int64, C.POINTER(OrMd),
            u32p, C.c_int64, C.c_int64, dp, dp, dp, C.POINTER(OrDeposit), C.c_int64, C.POINTER(C.c_int64),
        ]
        L.or_md_run.restype = C.c_int
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_philox4x32_10.restype = None
        L.or_uniform24.argtypes = [C.c_uint32]
        L.or_uniform24.restype = C.c_double
        L.or_md_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int, dp]
        L.or_md_normals.restype = None
        L.or_md_potential.argtypes = [C.POINTER(OrMd), dp, dp]
        L.or_md_potential.restype = C.c_double
        L.or_run.restype = C.c_int
        L.or_langevin_double_well.argtypes = [
            C.POINTER(OrWalker), dp, dp, C.c_int64, C.c_double, C.c_double, C.c_double, dp, dp,
        ]
        L.or_langevin_double_well.restype = C.c_int
        L.or_compact.argtypes = [C.c_double, C.c_double, C.c_int, dp]
        L.or_compact.restype = C.c_double
        L.or_deposit_compact.argtypes = [C.POINTER(OrGrid), C.POINTER(OrHill), dp, dp, C.c_double, ip, dp]
        L.or_deposit_compact.restype = None
        L.or_lookup_mabp.argtypes = [C.POINTER(OrGrid), C.POINTER(OrHill), dp, dp, dp, dp]
        L.or_lookup_mabp.restype = C.c_int
        L.or_num_threads.argtypes = []
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().or_num_threads())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class Walker:
    """Oracle view of one walker spec (keeps the arrays its struct points at)."""

    def __init__(self, spec: dict):
        self.spec = spec
        self._keep = []
        s = OrWalker()
        g, hl = spec["grid"], spec["hill"]
        d = len(g["n"])
        s.g.d = d
        for k in range(d):
            s.g.n[k] = int(g["n"][k])
            s.g.periodic[k] = int(bool(g["periodic"][k]))
            s.g.lo[k] = float(g["lo"][k])
            s.g.hi[k] = float(g["hi"][k])
        s.hill.w = float(hl["w"])
        s.hill.method = METHODS[hl.get("method", "wt")]
        if s.hill.method == METHODS["mabp"]:
            for k in range(d):
                s.hill.a[k] = float(hl["a"][k])
            s.hill.p = int(hl["p"])
            s.hill.b = float(hl["b"])
            s.hill.c = float(hl["c"])
        else:
            for k in range(d):
                s.hill.sigma[k] = float(hl["sigma"][k])
            s.hill.cutoff = float(hl["cutoff"])
            s.hill.gamma = float(hl["gamma"])
        s.hill.kT = float(hl["kT"])
        s.hill.stride = int(hl["stride"])
        if hl.get("kwall", 0.0) > 0:
            s.hill.kwall = float(hl["kwall"])
            for k in range(d):
                s.hill.smax[k] = float(hl["smax"][k])
        cvs = spec["cvs"]
        if len(cvs) != d:
            raise ValueError("one CV per grid axis")
        for k, cv in enumerate(cvs):
            c = s.cv[k]
            c.type = CV_TYPES[cv["type"]]
            a = np.ascontiguousarray(cv["a"], dtype=np.int32)
            b = np.ascontiguousarray(cv.get("b", np.zeros(0)), dtype=np.int32)
            self._keep += [a, b]
            c.na, c.nb = len(a), len(b)
            c.ia, c.ib = _iptr(a), _iptr(b)
            for key, field in (("ma", "ma"), ("mb", "mb")):
                m = cv.get(key)
                if m is not None:
                    m = np.ascontiguousarray(m, dtype=np.float64)
                    self._keep.append(m)
                    setattr(c, field, _dptr(m))
            c.r0 = float(cv.get("r0", 0.4))
            c.nn = int(cv.get("n", 6))
            c.mm = int(cv.get("m", 12))
            c.pbc = int(bool(cv.get("pbc", False)))
            box = cv.get("box", (0.0, 0.0, 0.0))
            for q in range(3):
                c.box[q] = float(box[q])
            if cv["type"] == "rmsd":
                ref = np.ascontiguousarray(cv["ref"], dtype=np.float64).reshape(len(a), 3)
                self._keep.append(ref)
                c.ref = _dptr(ref)
        s.natoms = int(spec["natoms"])
        self.struct = s
        self.d = d
        self.nodes = int(np.prod(g["n"]))
        rc = lib().or_check(C.byref(s.g), C.byref(s.hill))
        if rc:
            raise ValueError(f"oracle rejects walker spec (code {rc})")

    def new_field(self) -> np.ndarray:
        """Zeroed grid: [nodes][1+d], axis 0 fastest."""
        return np.zeros((self.nodes, 1 + self.d), dtype=np.float64)

    def halfwidth(self, k: int) -> int:
        return int(lib().or_stencil_halfwidth(C.byref(self.struct.g), C.byref(self.struct.hill), k))


# ---------------------------------------------------------------- low level


def cv_eval(walker: Walker, k: int, x: np.ndarray):
    """CV k of the walker at coordinates x (natoms, 3). Returns (s, J, flags)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    J = np.zeros_like(x)
    s = C.c_double()
    fl = lib().or_cv_eval(C.byref(walker.struct.cv[k]), walker.struct.natoms, _dptr(x), C.byref(s), _dptr(J))
    return s.value, J, fl


def switch(x: float, n: int = 6, m: int = 12):
    d = C.c_double()
    v = lib().or_switch(float(x), int(n), int(m), C.byref(d))
    return v, d.value


def interp(walker: Walker, field: np.ndarray, s):
    s3 = np.zeros(3)
    s3[: walker.d] = s
    V = C.c_double()
    dV = np.zeros(3)
    fl = lib().or_interp(C.byref(walker.struct.g), _dptr(field), _dptr(s3), C.byref(V), _dptr(dV))
    return V.value, dV[: walker.d].copy(), fl


def height(walker: Walker, Vb: float) -> float:
    return float(lib().or_height(C.byref(walker.struct.hill), float(Vb)))


def deposit(walker: Walker, field: np.ndarray, s, h: float):
    """Deposit one hill of height h at s into field (in place): a Gaussian
    for a well-tempered walker, a compact hill at the nearest node (scaled by
    h) for an mABP walker. Returns the centre node."""
    assert field.dtype == np.float64 and field.flags.c_contiguous
    s3 = np.zeros(3)
    s3[: walker.d] = s
    ic = np.zeros(3, dtype=np.int32)
    fn = lib().or_deposit_compact if walker.struct.hill.method == METHODS["mabp"] else lib().or_deposit_hill
    fn(C.byref(walker.struct.g), C.byref(walker.struct.hill), _dptr(field), _dptr(s3), float(h), _iptr(ic), None)
    return ic[: walker.d].copy()


def compact(u: float, a: float, p: int):
    """The one-dimensional compact hill S_a^p(u) and dS/du."""
    d = C.c_double()
    v = lib().or_compact(float(u), float(a), int(p), C.byref(d))
    return v, d.value


def lookup_mabp(walker: Walker, field: np.ndarray, s):
    """mABP bias V and dV/dxi at the nearest node to s. Returns (V, dV, flags)."""
    s3 = np.zeros(3)
    s3[: walker.d] = s
    V = C.c_double()
    dV = np.zeros(3)
    fl = lib().or_lookup_mabp(C.byref(walker.struct.g), C.byref(walker.struct.hill), _dptr(field), _dptr(s3),
                              C.byref(V), _dptr(dV))
    return V.value, dV[: walker.d].copy(), fl


# ---------------------------------------------------------------- replay


def run(walkers, frames, atom_offsets, step0: int, T: int, fields=None, record_forces=True,
        dep_cap: int | None = None, md: dict | None = None, streams=None, error_model: bool = False):
    """Open-loop replay of T steps (step0 .. step0+T-1) for a batch of walkers.

    walkers: list of Walker. frames: float array [T, total_atoms, 3] (any
    float dtype; upcast to float64 exactly). atom_offsets[w]: index of walker
    w's first atom in a frame. fields: list of per-walker grids (float64
    [nodes, 1+d]); walkers given the same array object share that grid. New
    zeroed grids are made when fields is None. Returns a dict with s, V, dV
    ([T, nw, 3] / [T, nw]), F ([T, total_atoms, 3] or None), flags, the deposit
    log and the final fields. With md (closed-loop dynamics, see md_struct)
    and streams (one noise stream per walker) it also returns Xn
    [T, total_atoms, 3]: for every step, the coordinates after that step's
    move predicted from the recorded frame. With error_model it also returns
    the per-step error-analysis outputs: H [T, nw, 3, 3] (slope of the
    interpolated dV_k along s_j), A [T, nw, 4] (the interpolated gross
    fields: the rounding scale of the accumulated grid and of the
    interpolation), sb [T, nw, 3] (CV rounding bound in units of the unit roundoff)
    and Jn [T, total_atoms, 3] (|ds_k/dx| per atom).
    """
    nw = len(walkers)
    frames = np.ascontiguousarray(frames, dtype=np.float64)
    assert frames.ndim == 3 and frames.shape[0] == T and frames.shape[2] == 3
    total = frames.shape[1]
    if fields is None:
        fields = [w.new_field() for w in walkers]
    for f in fields:
        assert f.dtype == np.float64 and f.flags.c_contiguous
    arr = (OrWalker * nw)(*[w.struct for w in walkers])
    fptrs = (C.POINTER(C.c_double) * nw)(*[_dptr(f) for f in fields])
    offs = np.ascontiguousarray(np.asarray(atom_offsets, dtype=np.int64) * 3)
    s = np.zeros((T, nw, 3))
    V = np.zeros((T, nw))
    dV = np.zeros((T, nw, 3))
    F = np.zeros((T, total, 3)) if record_forces else None
    flags = np.zeros((T, nw), dtype=np.int32)
    if dep_cap is None:
        dep_cap = sum(T // w.struct.hill.stride + 1 for w in walkers)
    deps = (OrDeposit * max(dep_cap, 1))()
    nd = C.c_int64()
    mds, st, Xn = None, None, None
    if md is not None:
        mds = md_struct(md)
        st = np.ascontiguousarray(np.asarray(streams, dtype=np.uint32))
        assert st.shape == (nw,)
        Xn = np.zeros((T, total, 3))
    aux = (OrStepAux * (T * nw))() if error_model else None
    Jn = np.zeros((T, total, 3)) if error_model else None
    gptrs = None
    if error_model:
        # gross fields, shared where the fields are
        by_id = {}
        for f in fields:
            by_id.setdefault(id(f), np.abs(f))  # what the grid already holds counts at its size
        gross = [by_id[id(f)] for f in fields]
        gptrs = (C.POINTER(C.c_double) * nw)(*[_dptr(g) for g in gross])
    rc = lib().or_run(
        nw, arr, fptrs, _dptr(frames), offs.ctypes.data_as(C.POINTER(C.c_int64)), total * 3, int(step0), int(T),
        _dptr(s), _dptr(V), _dptr(dV), _dptr(F) if F is not None else None, _iptr(flags), deps, dep_cap, C.byref(nd),
        C.byref(mds) if mds is not None else None, st.ctypes.data_as(C.POINTER(C.c_uint32)) if st is not None else None,
        _dptr(Xn) if Xn is not None else None, aux, _dptr(Jn) if Jn is not None else None, gptrs,
    )
    if rc:
        raise RuntimeError(f"oracle run failed ({rc})")
    n = min(nd.value, dep_cap)
    log = {
        "step": np.array([deps[i].step for i in range(n)], dtype=np.int64),
        "walker": np.array([deps[i].walker for i in range(n)], dtype=np.int32),
        "ic": np.array([list(deps[i].ic) for i in range(n)], dtype=np.int32).reshape(n, 3),
        "s": np.array([list(deps[i].s) for i in range(n)]).reshape(n, 3),
        "height": np.array([deps[i].height for i in range(n)]),
    }
    out = {"s": s, "V": V, "dV": dV, "F": F, "flags": flags, "deposits": log, "fields": fields, "Xn": Xn}
    if error_model:
        a = np.ctypeslib.as_array(aux).view(np.float64).reshape(T, nw, 16)
        out.update(H=a[:, :, 0:9].reshape(T, nw, 3, 3).copy(), A=a[:, :, 9:13].copy(), sb=a[:, :, 13:16].copy(),
                   Jn=Jn)
    return out


def langevin_double_well(walker: Walker, field: np.ndarray, x0: np.ndarray, T: int, dt: float, mu: float,
                         kw: float, noise: np.ndarray):
    """Closed-loop overdamped Langevin on U(s) = kw (s^2-1)^2 plus the bias.

    noise: [T, natoms, 3] standard normals. Returns (final x, s history)."""
    x = np.ascontiguousarray(x0, dtype=np.float64).copy()
    noise = np.ascontiguousarray(noise, dtype=np.float64)
    assert noise.shape == (T, walker.struct.natoms, 3)
    s_hist = np.zeros(T)
    rc = lib().or_langevin_double_well(C.byref(walker.struct), _dptr(field), _dptr(x), int(T), float(dt), float(mu),
                                       float(kw), _dptr(noise), _dptr(s_hist))
    if rc:
        raise RuntimeError(f"oracle langevin failed ({rc})")
    return x, s_hist


# ---------------------------------------------------------------- closed-loop dynamics


def philox4x32_10(ctr, key):
    """Philox-4x32-10 of a 4-word counter and a 2-word key (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    u32p = C.POINTER(C.c_uint32)
    lib().or_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
    return out


def uniform24(r: int) -> float:
    return float(lib().or_uniform24(int(r) & 0xFFFFFFFF))


def md_normals(seed: int, stream: int, step: int, atom: int) -> np.ndarray:
    """The three standard normals of one atom at one MD step."""
    n = np.zeros(3)
    lib().or_md_normals(int(seed) & ((1 << 64) - 1), int(stream), int(step), int(atom), _dptr(n))
    return n


def md_potential(md: dict, s):
    """U(s) and dU/ds of the closed-loop dynamics' CV potential."""
    m = md_struct(md)
    s3 = np.zeros(3)
    s3[: len(s)] = s
    dU = np.zeros(3)
    U = lib().or_md_potential(C.byref(m), _dptr(s3), _dptr(dU))
    return float(U), dU


def md_run(walkers, x0, atom_offsets, md: dict, streams, step0: int, T: int, fields=None, record_x=False,
           dep_cap: int | None = None):
    """Closed-loop run of T steps (step0 .. step0+T-1) from coordinates x0
    [total_atoms, 3]. Returns a dict with the final x, X (the coordinates each
    step's bias was evaluated at, [T, total_atoms, 3], when record_x), s, V,
    the deposit log and the fields."""
    nw = len(walkers)
    x = np.ascontiguousarray(x0, dtype=np.float64).copy()
    total = x.shape[0]
    if fields is None:
        fields = [w.new_field() for w in walkers]
    arr = (OrWalker * nw)(*[w.struct for w in walkers])
    fptrs = (C.POINTER(C.c_double) * nw)(*[_dptr(f) for f in fields])
    offs = np.ascontiguousarray(np.asarray(atom_offsets, dtype=np.int64) * 3)
    mds = md_struct(md)
    st = np.ascontiguousarray(np.asarray(streams, dtype=np.uint32))
    X = np.zeros((T, total, 3)) if record_x else None
    s = np.zeros((T, nw, 3))
    V = np.zeros((T, nw))
    if dep_cap is None:
        dep_cap = sum(T // w.struct.hill.stride + 1 for w in walkers)
    deps = (OrDeposit * max(dep_cap, 1))()
    nd = C.c_int64()
    rc = lib().or_md_run(nw, arr, fptrs, _dptr(x), offs.ctypes.data_as(C.POINTER(C.c_int64)), total * 3,
                         C.byref(mds), st.ctypes.data_as(C.POINTER(C.c_uint32)), int(step0), int(T),
                         _dptr(X) if X is not None else None, _dptr(s), _dptr(V), deps, dep_cap, C.byref(nd))
    if rc:
        raise RuntimeError(f"oracle md run failed ({rc})")
    n = min(nd.value, dep_cap)
    log = {
        "step": np.array([deps[i].step for i in range(n)], dtype=np.int64),
        "walker": np.array([deps[i].walker for i in range(n)], dtype=np.int32),
        "s": np.array([list(deps[i].s) for i in range(n)]).reshape(n, 3),
        "height": np.array([deps[i].height for i in range(n)]),
    }
    return {"x": x, "X": X, "s": s, "V": V, "deposits": log, "fields": fields}


# ---------------------------------------------------------------- error analysis (test tolerances)


def interp_aux(walker: Walker, field: np.ndarray, s):
    """Slopes H[k, j] = d(dV_k)/ds_j of the interpolant and its absolute scale A."""
    s3 = np.zeros(3)
    s3[: walker.d] = s
    H = np.zeros(9)
    A = np.zeros(4)
    lib().or_interp_aux(C.byref(walker.struct.g), _dptr(field), None, _dptr(s3), _dptr(H), _dptr(A))
    return H.reshape(3, 3)[: walker.d, : walker.d].copy(), A[: 1 + walker.d].copy()


def cv_round_bound(walker: Walker, k: int, x: np.ndarray) -> float:
    """First-order rounding bound of CV k at x, in units of the unit roundoff."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    return float(lib().or_cv_round_bound(C.byref(walker.struct.cv[k]), _dptr(x)))
