"""Seeded synthetic inputs: walker specs and coordinate frames.

This module holds no arithmetic of the biasing method (no CV, hill,
interpolation or force formula). It only places atoms and writes the
parameters of each workload as plain data, so both the CUDA path and the
FP64 oracle can consume the same inputs.

Walker spec (a dict):
    natoms : atoms in the walker's own block (CV atoms only)
    cvs    : one dict per CV / grid axis:
             {"type": "com_dist" | "dihedral" | "coord",
              "a": atom indices (group A / the 4 dihedral atoms / ligand),
              "b": atom indices (group B / -- / pocket or environment),
              "ma", "mb": optional masses, "r0", "n", "m": switching function,
              "pbc": minimum image on, "box": orthorhombic box edges (nm)}
    grid   : {"lo", "hi", "n", "periodic"} per axis (nodes, see the library)
    hill   : {"w", "sigma", "cutoff", "gamma", "kT", "stride"}
    shared : optional key; walkers with the same key share one grid

Units: nm, kJ/mol, rad. Frames are float32 [T, total_atoms, 3]; walker w owns
atoms offsets[w] .. offsets[w] + natoms - 1 of every frame.

Workload recipes. Each is a seeded stand-in for the MD trajectories the
paper's runs bias (a ligand in a protein pocket, described by centre-of-mass
distances, dihedrals, coordination numbers or RMSDs): no trajectory or
structure data is available, so atoms are drawn from simple geometric
templates with the same atom counts, CV kinds and grid sizes:
  * ``double_well_com``: 1 walker, two 8-atom groups in a 3 nm box,
    1D grid of 512 nodes on [-2, 2], sigma 0.05, w 1, stride 100, gamma 10.
  * ``mb64``: 64 walkers, COM distance of two 16-atom groups in [0.2, 2.0]
    plus a periodic dihedral, own 256 x 256 grid, sigma (0.04, 0.1), w 0.5,
    stride 50, gamma 15. Frames sweep the CV box along a smooth per-walker
    path with 0.02 nm Gaussian jitter per atom and frame.
  * ``uneven1000``: 1000 walkers of 440 atoms (40 ligand in a 0.5 nm ball,
    400 pocket in a 0.6-1.5 nm shell); 40 % 1D CN on 1024 nodes, 50 % 2D
    (COM distance, CN) on 128^2/256^2/512^2, 10 % 3D (COM distance, ligand
    dihedral, CN) on 64^3; sigma 2 bins, cutoff 4 sigma, w 0.5, stride 50,
    gamma 15; frames = template + N(0, 0.02^2).
  * ``serve4096``: simulations with 2D grids of side U{64..1024}, 8-256 atoms,
    stride U{20..500}, sigma 2 bins, w 0.5, gamma 15.
  * ``shared256``: 32 walkers on one shared 256^3 grid, 200 ligand + 10,000
    environment atoms uniform in a 6 nm periodic box; sigma 2 bins,
    cutoff 4 sigma, w 0.2, stride 10, gamma 20.
"""
from __future__ import annotations

import math

import numpy as np

KT_300K = 2.494  # kJ/mol at 300 K


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- geometry


def _ball(r: np.random.Generator, n: int, radius: float) -> np.ndarray:
    v = r.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    rad = radius * r.random(n) ** (1.0 / 3.0)
    return v * rad[:, None]


def _shell(r: np.random.Generator, n: int, r_in: float, r_out: float) -> np.ndarray:
    v = r.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    rad = (r_in ** 3 + (r_out ** 3 - r_in ** 3) * r.random(n)) ** (1.0 / 3.0)
    return v * rad[:, None]


def _unit(r: np.random.Generator) -> np.ndarray:
    v = r.normal(size=3)
    return v / np.linalg.norm(v)


def _frame_basis(r: np.random.Generator):
    """A random right-handed orthonormal basis (ex, ey, ez)."""
    ez = _unit(r)
    t = _unit(r)
    ex = t - ez * (t @ ez)
    ex /= np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    return ex, ey, ez


def grid(lo, hi, n, periodic):
    return {"lo": list(map(float, lo)), "hi": list(map(float, hi)), "n": list(map(int, n)),
            "periodic": list(map(bool, periodic))}


def hill(w, sigma, stride, gamma, kT=2.5, cutoff=4.0):
    return {"w": float(w), "sigma": list(map(float, sigma)), "cutoff": float(cutoff), "gamma": float(gamma),
            "kT": float(kT), "stride": int(stride)}


def mabp_hill(a, p, b, c, kT=2.5, stride=1, w=1.0):
    """Hill parameters of an mABP walker with compact S_a^p hills: half-width a
    per CV, shape exponent p, bias parameters b, c; hills of height w every
    `stride` steps."""
    return {"method": "mabp", "a": list(map(float, a)), "p": int(p), "b": float(b), "c": float(c),
            "kT": float(kT), "stride": int(stride), "w": float(w)}


def with_wall(hill: dict, smax, kwall: float) -> dict:
    """The hill parameters plus the CV range limit: a harmonic wall of force
    constant kwall above smax_k on each CV."""
    return dict(hill, smax=list(map(float, smax)), kwall=float(kwall))


def bins(g: dict, k: int, nbins: float) -> float:
    """Width of `nbins` grid spacings along axis k (the node convention)."""
    n = g["n"][k]
    L = g["hi"][k] - g["lo"][k]
    return nbins * (L / n if g["periodic"][k] else L / (n - 1))


def offsets_of(specs) -> np.ndarray:
    off = np.zeros(len(specs), dtype=np.int64)
    acc = 0
    for i, s in enumerate(specs):
        off[i] = acc
        acc += s["natoms"]
    return off


# ---------------------------------------------------------------- mb64 (two CVs, 36 atoms)


class SweepWalker:
    """Template for a 36-atom walker whose COM separation and dihedral follow
    a smooth seeded path (for a COM-distance + dihedral grid)."""

    def __init__(self, r: np.random.Generator, r_range=(0.3, 1.9), period=(2000, 8000), dihedral_period=(1500, 6000)):
        self.ga = _ball(r, 16, 0.3)
        self.ga -= self.ga.mean(axis=0)
        self.gb = _ball(r, 16, 0.3)
        self.gb -= self.gb.mean(axis=0)
        self.ca = 1.5 + 0.2 * r.normal(size=3)
        self.axis = _unit(r)
        lo, hi = r_range
        self.rc = 0.5 * (lo + hi)
        self.ra = 0.5 * (hi - lo)
        self.P = r.uniform(*period)
        self.phase = r.uniform(0, 2 * math.pi)
        self.ex, self.ey, self.ez = _frame_basis(r)
        self.p0 = self.ca + 0.8 * _unit(r)
        self.theta0 = r.uniform(-math.pi, math.pi)
        self.Pth = r.uniform(*dihedral_period) * (1 if r.random() < 0.5 else -1)
        self.bond = 0.15

    def at(self, t: np.ndarray) -> np.ndarray:
        """Template coordinates for steps t: [len(t), 36, 3]."""
        t = np.asarray(t, dtype=np.float64)
        T = t.shape[0]
        out = np.empty((T, 36, 3))
        rsep = self.rc + self.ra * np.sin(2 * math.pi * t / self.P + self.phase)
        cb = self.ca[None, :] + rsep[:, None] * self.axis[None, :]
        out[:, 0:16] = self.ca[None, None, :] + self.ga[None]
        out[:, 16:32] = cb[:, None, :] + self.gb[None]
        th = self.theta0 + 2 * math.pi * t / self.Pth
        x2 = self.p0
        x3 = self.p0 + self.bond * self.ez
        x1 = x2 + self.bond * self.ex
        out[:, 32] = x1
        out[:, 33] = x2
        out[:, 34] = x3
        out[:, 35] = x3[None, :] + self.bond * (np.cos(th)[:, None] * self.ex + np.sin(th)[:, None] * self.ey)
        return out


def mb64_specs(nw: int = 64, n=(256, 256), stride: int = 50, w: float = 0.5, gamma: float = 15.0,
               sigma=(0.04, 0.1), kT: float = 2.5, cutoff: float = 4.0):
    g = grid((0.2, -math.pi), (2.0, math.pi), n, (False, True))
    spec = {
        "natoms": 36,
        "cvs": [
            {"type": "com_dist", "a": np.arange(0, 16), "b": np.arange(16, 32)},
            {"type": "dihedral", "a": np.arange(32, 36)},
        ],
        "grid": g,
        "hill": hill(w, sigma, stride, gamma, kT, cutoff),
    }
    return [dict(spec) for _ in range(nw)]


class SweepFrames:
    """Open-loop frames for walkers built from SweepWalker templates."""

    def __init__(self, nw: int, seed: int, jitter: float = 0.02, **kw):
        r = rng(seed)
        self.walkers = [SweepWalker(r, **kw) for _ in range(nw)]
        self.jitter = jitter
        self.seed = seed

    def frames(self, step0: int, T: int, dtype=np.float32) -> np.ndarray:
        t = np.arange(step0, step0 + T)
        tmpl = np.concatenate([w.at(t) for w in self.walkers], axis=1)
        noise = rng(self.seed * 1_000_003 + step0 + 17).normal(scale=self.jitter, size=tmpl.shape)
        return (tmpl + noise).astype(dtype)


# ---------------------------------------------------------------- closed-loop dynamics (plain data)

# The four-term surface of Mueller and Brown (Theor. Chim. Acta 53, 1979):
# U(X, Y) = sum_i A_i exp(a_i (X - x0_i)^2 + b_i (X - x0_i)(Y - y0_i) + c_i (Y - y0_i)^2).
MULLER_BROWN = {"A": (-200.0, -100.0, -170.0, 15.0), "a": (-1.0, -1.0, -6.5, 0.7), "b": (0.0, 0.0, 11.0, 0.6),
                "c": (-10.0, -10.0, -6.5, 0.7), "x0": (1.0, 0.0, -0.5, -1.0), "y0": (0.0, 0.5, 1.5, 1.0)}


def md_params(dt: float = 0.002, mu: float = 1.0, kT: float = 2.5, seed: int = 1, potential: str = "none", **kw):
    """Closed-loop dynamics: overdamped Langevin of every CV atom, time step
    dt (ps), mobility mu (nm^2 / (kJ/mol ps)), noise at kT, Philox key seed,
    under the bias plus an optional potential of the CVs."""
    p = {"dt": float(dt), "mu": float(mu), "kT": float(kT), "seed": int(seed), "potential": potential}
    p.update(kw)
    return p


def md_double_well(seed: int = 1, A: float = 5.0, B: float = 1.0, **kw):
    """U(s) = A (s_0^2 - B^2)^2 on the first CV (A = 5 kJ/mol, B = 1 nm)."""
    return md_params(seed=seed, potential="double_well", dw=(float(A), float(B)), **kw)


def md_muller_brown(seed: int = 1, s_box=((0.2, 2.0), (-math.pi, math.pi)), xy_box=((-1.5, 1.2), (-0.2, 2.0)),
                    scale: float = 0.1, mu: float = 0.1, **kw):
    """The Mueller-Brown surface times `scale` on the affine image of the CV
    box s_box onto xy_box (X = mx s_0 + cx, Y = my s_1 + cy)."""
    (s0a, s0b), (s1a, s1b) = s_box
    (xa, xb), (ya, yb) = xy_box
    mx = (xb - xa) / (s0b - s0a)
    my = (yb - ya) / (s1b - s1a)
    mb = dict(MULLER_BROWN, scale=float(scale), map=(mx, xa - mx * s0a, my, ya - my * s1a))
    return md_params(seed=seed, potential="muller_brown", mb=mb, mu=mu, **kw)


# ---------------------------------------------------------------- double well (one walker, FP64)


def double_well_com_spec(n: int = 512, sigma: float = 0.05, w: float = 1.0, stride: int = 100, gamma: float = 10.0,
                         kT: float = 2.5):
    return {
        "natoms": 16,
        "cvs": [{"type": "com_dist", "a": np.arange(0, 8), "b": np.arange(8, 16)}],
        "grid": grid((-2.0,), (2.0,), (n,), (False,)),
        "hill": hill(w, (sigma,), stride, gamma, kT),
    }


def double_well_com_coords(seed: int) -> np.ndarray:
    """Two 8-atom groups seeded uniform in a 3 nm box: [16, 3] float64."""
    return rng(seed).uniform(0.0, 3.0, size=(16, 3))


# ---------------------------------------------------------------- ligand / pocket templates


def ligand_pocket_template(r: np.random.Generator, n_lig: int = 40, n_pocket: int = 400,
                           offset: float = 0.3) -> np.ndarray:
    lig = _ball(r, n_lig, 0.5) + offset * _unit(r)
    poc = _shell(r, n_pocket, 0.6, 1.5)
    return np.concatenate([lig, poc], axis=0) + 2.0


# Coordination-number axis ranges (count units). The template recipes put the
# ligand-pocket CN well inside these ranges; a test checks this with the
# oracle for the seeds used.
CN_RANGE_UNEVEN = (80.0, 480.0)
CN_RANGE_SHARED = (3000.0, 5000.0)


def uneven1000_specs(seed: int, nw: int = 1000, stride: int = 50, w: float = 0.5, gamma: float = 15.0,
                     kT: float = 2.5, n_lig: int = 40, n_pocket: int = 400, sizes_2d=(128, 256, 512),
                     n1d: int = 1024, n3d: int = 64):
    """Specs for the uneven batch (40 % 1D, 50 % 2D, 10 % 3D, shuffled)."""
    r = rng(seed)
    nat = n_lig + n_pocket
    lig = np.arange(0, n_lig)
    poc = np.arange(n_lig, nat)
    cn = {"type": "coord", "a": lig, "b": poc, "r0": 0.4, "n": 6, "m": 12}
    dist = {"type": "com_dist", "a": lig, "b": poc}
    dih = {"type": "dihedral", "a": np.arange(0, 4)}
    kinds = np.array([1] * int(round(0.4 * nw)) + [2] * int(round(0.5 * nw)) + [3] * (nw - int(round(0.4 * nw)) - int(round(0.5 * nw))))
    r.shuffle(kinds)
    specs = []
    for kd in kinds:
        if kd == 1:
            g = grid((CN_RANGE_UNEVEN[0],), (CN_RANGE_UNEVEN[1],), (n1d,), (False,))
            cvs = [cn]
        elif kd == 2:
            side = int(r.choice(sizes_2d))
            g = grid((0.0, CN_RANGE_UNEVEN[0]), (2.0, CN_RANGE_UNEVEN[1]), (side, side), (False, False))
            cvs = [dist, cn]
        else:
            g = grid((0.0, -math.pi, CN_RANGE_UNEVEN[0]), (2.0, math.pi, CN_RANGE_UNEVEN[1]), (n3d,) * 3,
                     (False, True, False))
            cvs = [dist, dih, cn]
        sig = [bins(g, k, 2.0) for k in range(len(cvs))]
        specs.append({"natoms": nat, "cvs": cvs, "grid": g, "hill": hill(w, sig, stride, gamma, kT)})
    return specs


class JitterFrames:
    """Frames = fixed per-walker template + N(0, jitter^2) per atom and frame."""

    def __init__(self, templates, seed: int, jitter: float = 0.02):
        self.tmpl = np.concatenate(templates, axis=0)
        self.seed = seed
        self.jitter = jitter

    def frames(self, step0: int, T: int, dtype=np.float32) -> np.ndarray:
        noise = rng(self.seed * 1_000_003 + step0 + 29).normal(scale=self.jitter, size=(T,) + self.tmpl.shape)
        return (self.tmpl[None] + noise).astype(dtype)


def uneven1000_templates(seed: int, nw: int = 1000, **kw):
    r = rng(seed + 7)
    return [ligand_pocket_template(r, **kw) for _ in range(nw)]


# ---------------------------------------------------------------- serving (2D, 8-256 atoms)


def serve_specs(seed: int, nsim: int = 4096, side=(64, 1024), atoms=(8, 256), stride=(20, 500), w: float = 0.5,
                gamma: float = 15.0, kT: float = 2.5):
    """One spec per simulation: COM distance of the two halves of its atoms
    plus the dihedral of atoms 0-3, on a square grid."""
    r = rng(seed)
    specs = []
    for _ in range(nsim):
        s = int(r.integers(side[0], side[1] + 1))
        na = int(r.integers(atoms[0], atoms[1] + 1))
        half = na // 2
        g = grid((0.0, -math.pi), (2.5, math.pi), (s, s), (False, True))
        cvs = [{"type": "com_dist", "a": np.arange(0, half), "b": np.arange(half, na)},
               {"type": "dihedral", "a": np.arange(0, 4)}]
        sig = [bins(g, 0, 2.0), bins(g, 1, 2.0)]
        specs.append({"natoms": na, "cvs": cvs, "grid": g,
                      "hill": hill(w, sig, int(r.integers(stride[0], stride[1] + 1)), gamma, kT)})
    return specs


def serve_templates(seed: int, specs):
    r = rng(seed + 11)
    out = []
    for s in specs:
        na = s["natoms"]
        half = na // 2
        a = _ball(r, half, 0.4)
        b = _ball(r, na - half, 0.4) + (0.5 + 1.2 * r.random()) * _unit(r)
        out.append(np.concatenate([a, b]) + 2.0)
    return out


# ---------------------------------------------------------------- shared 256^3 grid


def shared256_specs(nw: int = 32, n: int = 256, n_lig: int = 200, n_env: int = 10_000, box: float = 6.0,
                    stride: int = 10, w: float = 0.2, gamma: float = 20.0, kT: float = 2.5,
                    cn_range=CN_RANGE_SHARED):
    nat = n_lig + n_env
    lig = np.arange(0, n_lig)
    env = np.arange(n_lig, nat)
    bx = (box, box, box)
    # the minimum-image COM distance in a cubic box of edge L is at most L*sqrt(3)/2
    g = grid((0.0, -math.pi, cn_range[0]), (box * math.sqrt(3.0) / 2.0, math.pi, cn_range[1]),
             (n, n, n), (False, True, False))
    cvs = [{"type": "com_dist", "a": lig, "b": env[:16], "pbc": True, "box": bx},
           {"type": "dihedral", "a": np.arange(0, 4), "pbc": True, "box": bx},
           {"type": "coord", "a": lig, "b": env, "r0": 0.4, "n": 6, "m": 12, "pbc": True, "box": bx}]
    sig = [bins(g, k, 2.0) for k in range(3)]
    spec = {"natoms": nat, "cvs": cvs, "grid": g, "hill": hill(w, sig, stride, gamma, kT), "shared": "shared256"}
    return [dict(spec) for _ in range(nw)]


def shared256_templates(seed: int, nw: int = 32, n_lig: int = 200, n_env: int = 10_000, box: float = 6.0):
    r = rng(seed + 13)
    out = []
    for _ in range(nw):
        lig = _ball(r, n_lig, 0.6) + r.uniform(0.5, box - 0.5, size=3)
        env = r.uniform(0.0, box, size=(n_env, 3))
        out.append(np.concatenate([lig, env]))
    return out


# ---------------------------------------------------------------- the paper's RMSD setup (mABP, 480^2 grid)


def paper_rmsd_specs(nw: int = 64, n: int = 480, lo: float = 0.0, hi: float = 12.0, a_bins: float = 10.0,
                     p: int = 20, b: float = 0.9, c: float = 0.001, kT: float = 2.5, stride: int = 1,
                     seed: int = 11):
    """Walkers shaped like the paper's ligand runs: two RMSD CVs (4 atoms
    each, to seeded reference positions) on a 480 x 480 grid over [0, 12] nm,
    mABP with compact hills a = 10 grid spacings, p = 20, b = 0.9, c = 0.001,
    updated every step."""
    r = rng(seed)
    g = grid((lo, lo), (hi, hi), (n, n), (False, False))
    a = [bins(g, k, a_bins) for k in range(2)]
    specs = []
    for _ in range(nw):
        ref = _ball(r, 8, 0.4)
        cvs = [{"type": "rmsd", "a": np.arange(0, 4), "ref": ref[:4].copy()},
               {"type": "rmsd", "a": np.arange(4, 8), "ref": ref[4:].copy()}]
        specs.append({"natoms": 8, "cvs": cvs, "grid": g, "hill": mabp_hill(a, p, b, c, kT, stride)})
    return specs


class RmsdFrames:
    """Frames for paper_rmsd_specs walkers: each 4-atom group is its reference
    shifted along a slow closed path (its RMSD sweeps about 0.1 to 3 nm over
    `period` steps: by default tens of thousands, a drift far slower than the
    atoms' N(0, jitter^2) vibration, as for a ligand's pose in MD)."""

    def __init__(self, specs, seed: int, amp=(0.3, 3.0), period=(20_000, 80_000), jitter: float = 0.02):
        r = rng(seed)
        self.ref = np.concatenate([np.concatenate([c["ref"] for c in sp["cvs"]]) for sp in specs])  # [nw*8, 3]
        ng = 2 * len(specs)
        self.amp = r.uniform(amp[0], amp[1], size=(ng, 3)) / math.sqrt(3.0)
        self.per = r.uniform(period[0], period[1], size=(ng, 3))
        self.phase = r.uniform(0, 2 * math.pi, size=(ng, 3))
        self.seed = seed
        self.jitter = jitter

    def frames(self, step0: int, T: int, dtype=np.float32) -> np.ndarray:
        t = np.arange(step0, step0 + T, dtype=np.float64)[:, None, None]
        shift = self.amp[None] * np.sin(2 * math.pi * t / self.per[None] + self.phase[None])  # [T, ng, 3]
        shift = np.repeat(shift, 4, axis=1)
        noise = rng(self.seed * 1_000_003 + step0 + 31).normal(scale=self.jitter, size=(T,) + self.ref.shape)
        return (self.ref[None] + shift + noise).astype(dtype)
