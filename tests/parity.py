"""Comparison helpers for the GPU-vs-oracle parity tests.

Error measures (all normwise):
  grid field q:  max_nodes |F_gpu - F_ref| / max_nodes |F_ref|
  V_b(s_t):      max_steps |V_gpu - V_ref| / max_steps |V_ref|
  forces:        max_steps max_atoms |F_gpu - F_ref| / max_steps max_atoms |F_ref|
                 (normwise over the trajectory: the force scale of a run is set
                 by the bias gradient, and on a step whose own force is small
                 the FP32 CV value -- about 1e-7 from the FP64 one, read where a
                 just-deposited hill has its largest curvature h / sigma^2 --
                 can make the step-local relative error exceed 1e-4 although
                 the absolute error is ~1e-6 of the force scale)
Tolerances (the target the build is held to): 1e-5 on V_b and the grid
fields, 1e-4 on atom forces.

Tie band: the hill centre index i_c = floor(u + 1/2) is decided from s_t,
which the GPU computes in FP32 terms and the oracle in FP64. When the
oracle's u lies within TIE_BAND of a half-integer both indices are valid;
the deposit is then counted as a tie and that walker is compared only on
what does not depend on the choice (its CV values).
"""
import numpy as np

TOL_V = 1e-5
TOL_F = 1e-4
TIE_BAND = 1e-4


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


def compare_deposits(specs, gpu_log, ref_log, id_to_index):
    """Match deposits by (walker, step); integer centres must agree outside
    the tie band. Returns the set of walker indices with a tie."""
    ref = {(int(w), int(st)): i for i, (w, st) in enumerate(zip(ref_log["walker"], ref_log["step"]))}
    assert len(gpu_log["step"]) == len(ref_log["step"]), (len(gpu_log["step"]), len(ref_log["step"]))
    ties = set()
    for j in range(len(gpu_log["step"])):
        w = id_to_index[int(gpu_log["walker_id"][j])]
        key = (w, int(gpu_log["step"][j]))
        assert key in ref, key
        i = ref[key]
        d = len(specs[w]["grid"]["n"])
        ic_g = gpu_log["ic"][j][:d]
        ic_r = ref_log["ic"][i][:d]
        if not np.array_equal(ic_g, ic_r):
            u = grid_u(specs[w], ref_log["s"][i])
            frac = np.abs((u % 1.0) - 0.5)
            bad = ic_g != ic_r
            assert np.all(frac[bad] < TIE_BAND), (key, ic_g, ic_r, u)
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
    """Per-step normwise error (reported, not gated; see above)."""
    nr = np.linalg.norm(Fref, axis=-1).max(axis=-1)
    ne = np.linalg.norm(F - Fref, axis=-1).max(axis=-1)
    return ne / np.maximum(nr, 1e-300)
