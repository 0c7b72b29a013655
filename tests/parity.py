"""Comparison helpers for the GPU-vs-oracle parity tests.

Error measures:
  grid field q:  max_nodes |F_gpu - F_ref| / max_nodes |F_ref|        (normwise)
  forces, run:   max_steps max_atoms |F_gpu - F_ref| / max_steps max_atoms |F_ref|
  forces, step:  at every step t and atom i
                   |F_gpu,i(t) - F_ref,i(t)| <= TOL_F max_j |F_ref,j(t)| + floor_i(t)
  CVs:           at every deposit, |s_gpu - s_ref| <= u sb (the CV's rounding bound)
Tolerances (the target the build is held to): 1e-5 on V_b and the grid
fields, 1e-4 on atom forces.

The per-step floor is the FP32 error model of the force, computed from the
oracle's own quantities at the step (oracle.run(..., error_model=True)):
  floor_i(t) = sum_k |ds_k/dx_i| (sum_j |d(dV_k)/ds_j| u sb_j + 16 u A_k).
The first term is what a CV error within its rounding bound u sb_j does to
the interpolated gradient (the slope of the interpolant times the CV
error); the second is the rounding of the grid and of the interpolation:
A_k interpolates the gross value of field k at the corners (the sum of the
absolute values of every hill's contribution there, each computed in FP32
to a few roundings of its size, where the derivative fields of overlapping
hills cancel), and the weights, products and corner sums cost at most
2d + 3 roundings, the force's products and sums d + 1 more, the Jacobian a
few; a last term of 2^-120
(FP32; 2^-1000 for FP64) stands for values below the format's normal range,
which the GPU's products flush (the compact hills of mABP reach e^-160 near
their support's edge). On a step whose own force
is tiny (a walker at the top or bottom of its bias, or at the centre of the
hill it just deposited) the relative tolerance alone would ask for more
digits than the FP32 CV carries; the floor is what FP32 CVs cannot avoid.

Tie band (integer pieces): the hill centre index i_c = floor(u + 1/2) is
decided from s_t, which the GPU computes in FP32 terms and the oracle in
FP64. Where the two indices differ, the oracle's u must lie within
4 |u_gpu - u_ref| + 1e-6 of a half-integer (both choices are then valid);
the deposit is counted as a tie and that walker is compared only on what
does not depend on the choice.
"""
import json
import os

import numpy as np

TOL_V = 1e-5
TOL_F = 1e-4
U32 = 2.0 ** -24
U64 = 2.0 ** -53
# Values below these underflow the format's normal range (2^-126, 2^-1022)
# somewhere in their products: a force of that size is zero to the GPU.
TINY = {U32: 2.0 ** -120, U64: 2.0 ** -1000}


def grid_u(spec, s):
    g = spec["grid"]
    u = []
    for k in range(len(g["n"])):
        n = g["n"][k]
        L = g["hi"][k] - g["lo"][k]
        D = L / n if g["periodic"][k] else L / (n - 1)
        uk = (s[k] - g["lo"][k]) / D
        if g["periodic"][k]:
            uk = uk % n
        u.append(uk)
    return np.array(u)


def compare_deposits(specs, gpu_log, ref_log, id_to_index, sb=None, unit=U32, step0=0):
    """Match deposits by (walker, step); integer centres must agree outside
    the tie band; with sb ([T, nw, 3] rounding bounds from the oracle's
    error model) every deposit's CV values are checked against it. Returns
    the set of walker indices with a tie."""
    ref = {(int(w), int(st)): i for i, (w, st) in enumerate(zip(ref_log["walker"], ref_log["step"]))}
    assert len(gpu_log["step"]) == len(ref_log["step"]), (len(gpu_log["step"]), len(ref_log["step"]))
    ties = set()
    for j in range(len(gpu_log["step"])):
        w = id_to_index[int(gpu_log["walker_id"][j])]
        key = (w, int(gpu_log["step"][j]))
        assert key in ref, key
        i = ref[key]
        d = len(specs[w]["grid"]["n"])
        s_g, s_r = gpu_log["s"][j][:d], ref_log["s"][i][:d]
        if sb is not None:
            bound = unit * sb[key[1] - step0, w, :d]
            assert np.all(np.abs(s_g - s_r) <= bound), (key, s_g - s_r, bound)
        ic_g = gpu_log["ic"][j][:d]
        ic_r = ref_log["ic"][i][:d]
        if not np.array_equal(ic_g, ic_r):
            u_r = grid_u(specs[w], s_r)
            u_g = grid_u(specs[w], s_g)
            du = np.abs(u_g - u_r)
            frac = np.abs((u_r % 1.0) - 0.5)
            bad = ic_g != ic_r
            assert np.all(frac[bad] < 4 * du[bad] + 1e-6), (key, ic_g, ic_r, u_r, du)
            ties.add(w)
        # heights agree unless an earlier tie changed this walker's grid
        if w not in ties:
            h_g, h_r = gpu_log["height"][j], ref_log["height"][i]
            assert abs(h_g - h_r) <= 1e-6 * abs(h_r), (key, h_g, h_r)
    return ties


def rel_field_err(a, ref):
    """Normwise error per field column."""
    den = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    return np.abs(a - ref).max(axis=0) / den


def force_err(F, Fref):
    """Normwise force error over a trajectory ([T, atoms, 3] arrays)."""
    nr = np.linalg.norm(Fref, axis=-1).max()
    ne = np.linalg.norm(F - Fref, axis=-1).max()
    return ne / max(nr, 1e-300)


def force_err_per_step(F, Fref):
    """Per-step normwise error: max_i |dF_i(t)| / max_i |F_ref,i(t)|."""
    nr = np.linalg.norm(Fref, axis=-1).max(axis=-1)
    ne = np.linalg.norm(F - Fref, axis=-1).max(axis=-1)
    return ne / np.maximum(nr, 1e-300)


def force_floor(ref, w, sl, d, unit=U32):
    """floor_i(t) of walker w (atoms sl, d CVs), [T, atoms] (see the module
    docstring)."""
    H = np.abs(ref["H"][:, w, :d, :d])
    ds = unit * ref["sb"][:, w, :d]
    A = ref["A"][:, w, 1:1 + d]
    E = np.einsum("tkj,tj->tk", H, ds) + 16.0 * unit * A + TINY[unit]
    return np.einsum("tak,tk->ta", ref["Jn"][:, sl, :d], E) + TINY[unit]


def check_forces_per_step(F, ref, w, sl, d, tol=TOL_F, unit=U32):
    """Gate the per-step force error of walker w; returns (worst per-step
    relative error, worst ratio of the error to its allowance, steps where
    the floor was needed)."""
    Fr = ref["F"][:, sl]
    err = np.linalg.norm(F[:, sl] - Fr, axis=-1)  # [T, atoms]
    scale = np.linalg.norm(Fr, axis=-1).max(axis=-1, keepdims=True)  # [T, 1]
    allow = tol * scale + force_floor(ref, w, sl, d, unit)
    ratio = err / np.maximum(allow, 1e-300)
    t, i = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio.max() <= 1.0, (w, int(t), int(i), float(err[t, i]), float(scale[t, 0]), float(allow[t, i]))
    rel = (err.max(axis=-1) / np.maximum(scale[:, 0], 1e-300))
    return float(rel.max()), float(ratio.max()), int(np.sum(rel > tol))


def record_errors(config, test, worst):
    """Append one test's worst errors to the JSON-lines file named by the
    ABP_ERROR_TABLE environment variable (nothing when it is unset): the
    per-configuration error table is assembled from these records."""
    path = os.environ.get("ABP_ERROR_TABLE")
    if not path:
        return
    row = {"config": config, "test": test}
    row.update({k: (float(v) if isinstance(v, (float, np.floating)) else v) for k, v in worst.items()})
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")
