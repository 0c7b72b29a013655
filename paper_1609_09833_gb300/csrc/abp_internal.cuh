// abp_internal.cuh -- device-side descriptors shared by the library's
// translation units (never exposed through include/abp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "abp.h"

namespace abp {

constexpr int kMaxCv = 3;
constexpr int kRMax = 64;            // largest stencil half-width per axis
constexpr int kMaxGroupWarps = 8;    // threads per walker group <= 256
constexpr int kMaxGroupsPerCta = 8;  // named barriers 1..8

// COM weights, index lists and switching parameters of one CV (device).
struct CvDev {
  int type;
  int na, nb;
  const int32_t *ia, *ib;      // device index lists (unique within a list)
  const float *wa, *wb;        // COM weights m_i / M_group (FP32 walkers)
  const double *wa64, *wb64;   // COM weights (FP64 walkers)
  double inv_r0sq;             // COORD: 1 / r0^2
  const float *ref;            // RMSD: reference positions (3 per atom of ia), FP32 walkers
  const double *ref64;         //       and FP64 walkers
  int pbc;
  double box[3];
  double inv_box[3];
  int hp;  // DIHEDRAL of an FP32 walker: the angle formed in FP64, carried as hi + lo
  // COM_DIST: relative error of the FP32 weights when a group's masses are
  // all equal (W / float(W) - 1, W = 1 / n), else 0; the FP32 finish scales
  // the group's weighted sum by 1 + wc
  float wc_a, wc_b;
};

struct GridDev {
  int d;
  int n[3];
  int periodic[3];
  double lo[3];
  double D[3];       // node spacing
  double invD[3];
  double L[3];       // axis length (periodic wrap)
  double u0[3];      // -lo / D: u = s * invD + u0
  double inv_n[3];   // 1 / n
  float invD_h[3], invD_l[3];  // invD and u0 as hi + lo floats (FP32 grids)
  float u0_h[3], u0_l[3];
  int prec;          // ABP_PREC_*
  int rec_bytes;     // bytes per node record
  long long nodes;
  void *rec;         // node records (see GridLayout below)
  int shared;        // several walkers deposit per step (see shadow)
  double *shadow;    // shared grids: FP64 accumulator, 4 doubles per node {V, dV0, dV1, dV2}
  unsigned long long *oob;  // checked builds: the context's count of out-of-grid node indices
};

// Node record layouts:
//   FP32_COMP, d = 1 : float4 {V, dV0, cV, cdV0}                     (16 B)
//   FP32_COMP, d > 1 : float4 {V, dV0, dV1, dV2|0} + float4 {cV, ...} (32 B)
//   FP64,      d = 1 : double {V, dV0}                               (16 B)
//   FP64,      d > 1 : double {V, dV0, dV1, dV2|0}                   (32 B)
// "c" = two-sum compensation: the field's value is sum + comp.

struct WalkerState {
  double s[3];
  double V;
  double dV[3];
  int flags;
  int pad;
  long long step;
};

struct WalkerDev {
  GridDev g;
  CvDev cv[kMaxCv];
  int natoms;
  int id;
  int R[3];          // stencil half-widths
  double sigma[3];
  double inv2s2[3];  // 1 / (2 sigma^2)
  double invs2[3];   // 1 / sigma^2
  double w;
  double inv_dT;     // 1 / ((gamma - 1) kT)
  long long stride;
  int method;        // ABP_METHOD_*
  int p;             // mABP: compact hill exponent
  double a[3];       // mABP: compact hill half-width per CV
  double mabp_k;     // mABP: kT b / (1 - b)   (Eq. (apfm): V = mabp_k ln(mabp_h h + 1))
  double mabp_g;     // mABP: c b kT           (Eq. (btraj-grad): dV = mabp_g h' / (1 + mabp_h h))
  double mabp_h;     // mABP: c (1 - b)
  double smax[3];    // CV range limit: wall above smax_k ...
  double kwall;      // ... of force constant kwall (0: none)
  float smax_f[3];   // the same in FP32 (the FP32 kernels' copies)
  float kwall_f;
  void *fbuf;        // library-owned force records (abp_step -> abp_forces)
  void *jscratch;    // library-owned Jacobian scratch (plain form)
  WalkerState *state;
  // a5 term tables of the closed-loop form, built at walker creation (or
  // null): per atom its count and kAtomTerms AtomTerm<Real> records, in CV
  // order, list A before list B
  const int *acnt;
  const void *aterms;
};

// Closed-loop dynamics of abp_md_run (device copy of abp_md_desc, with the
// move's two constants formed on the host in FP64).
struct MdParams {
  int potential;                 // ABP_POT_*
  int pad;
  double c1;                     // dt * mobility
  double c2;                     // sqrt(2 mobility kT dt)
  unsigned long long seed;
  double dw_a, dw_b;
  double mb_scale;
  double mb_map[4];
  double mb_A[4], mb_a[4], mb_b[4], mb_c[4], mb_x0[4], mb_y0[4];
};

// Deposit log (device side).
struct DepositLog {
  abp_deposit_rec *rec;
  unsigned long long *count;
  unsigned long long cap;
};

// Context-wide device counters.
struct DevCounters {
  int nonfinite;
  int pad0;
  unsigned long long oob;  // checked builds (ABP_CHECKED): node indices found outside their grid
  int pad[28];
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }
__host__ __device__ inline int align32(int x) { return (x + 31) & ~31; }

// One MD step of a window of the windowed form (shared memory): the step's
// CVs, Jacobian factors, axis state and interpolated bias.
template <typename Real>
struct StepRec {
  Real s[kMaxCv];         // CV values (FP32 walkers: the high part of a COM distance ...
  Real sl[kMaxCv];        // ... whose low part is here; 0 for the other CVs)
  Real jac[kMaxCv][12];   // COM distance: unit separation (3); dihedral, RMSD: gradient (4 x 3)
  Real f[kMaxCv];         // interpolation weight of i1
  Real df[kMaxCv];        // deposit: u - da
  Real V;                 // V_b(s) after the step's deposits
  Real dv[kMaxCv];        // dV_b/ds_k (0 on a clamped axis)
  int i0[kMaxCv], i1[kMaxCv];
  int da[kMaxCv], dc[kMaxCv], ic_log[kMaxCv];
  int cfl[kMaxCv];        // per CV: ABP_WFLAG_SINGULAR, and bit 16 if the axis is clamped
  int clamped;            // interpolation clamp mask
  int flags;              // ABP_WFLAG_*
};

// One term of an atom's a5 in the windowed form: f += w v, v the 3-vector at
// jac[0][0] + off of the step's record (a CV's Jacobian factor, scaled by
// dV_b/ds_k once the step is interpolated).
template <typename Real>
struct AtomTerm {
  Real w;
  int off;
};

constexpr int kWinMax = 32;             // MD steps per window of the windowed form
constexpr int kAtomTerms = 2 * kMaxCv;  // per atom: up to 2 list entries per CV
// FP32 walkers form a dihedral's angle in FP64 when its hill (WT: sigma;
// mABP: a) is narrower than this (rad): the FP32 angle's rounding, up to
// ~1.2e-7 rad near +-pi, would otherwise move the hill by 2e-6 of its width
// or more, against a 1e-5 tolerance on the grid fields.
constexpr double kDihedralHpWidth = 0.06;
constexpr int kMabpBoxBytes = 96 * 1024;  // windowed mABP: the union of a window's stencil boxes, at most
constexpr int kWinBytes = 64 * 1024;    // its coordinate double buffer, at most
constexpr int kWtBoxBytes = 64 * 1024;  // windowed WT: a deposit's stencil box, at most

// Steps per window for a walker in the windowed form (0: not eligible). The
// form takes walkers whose CVs are all COM distances, dihedrals or RMSDs of at
// most 4 atoms (one thread evaluates a step's CVs, and a step's Jacobian
// factors fit its record); the window's coordinates are double buffered in
// rows of natoms | 1 records (an odd row stride keeps the threads of a warp,
// one row each, on distinct banks).
__host__ __device__ inline int window_steps(int natoms, const CvDev *cv, int d, int rsz) {
  for (int k = 0; k < d; ++k)
    if (cv[k].type != ABP_CV_COM_DIST && cv[k].type != ABP_CV_DIHEDRAL &&
        !(cv[k].type == ABP_CV_RMSD && cv[k].na <= 4))
      return 0;
  const long long row = (long long)(natoms | 1) * rsz;
  for (int W = kWinMax; W >= 4; W >>= 1)
    if (2 * W * row <= kWinBytes) return W;
  return 0;
}

// Shared-memory layout of one walker group (computed identically on host and
// device). Offsets are bytes from the start of the group's dynamic part.
//   xs0, xs1  coordinates of two steps (the next step's arrive by cp.async);
//             in the windowed form, of two windows of `win` steps, rows of
//             `xstride` records (the current window's rows then hold its
//             force accumulators)
//   fs        force accumulators (per-step form)
//   steps     StepRec arrays of the three windows in flight (windowed form)
//   atoms     per atom, its a5 terms: counts, then AtomTerm[natoms][kAtomTerms] (windowed form)
//   lists     per-CV atom index lists (+ COM weights)
//   cn        per COORD CV: dCN/dx per list entry and per-warp partials
//   tile      optional copy of a box of the walker's grid (node records); in
//             the windowed form, a deposit's stencil box (WT walkers of 1 or 2
//             CVs whose box has at most one node per chain-half thread) or
//             the union of a window's boxes (mABP)
struct GroupLayout {
  int xs0, xs1, fs, steps, atoms, lists, cn, tile, total;
  int win, xstride;  // windowed form: steps per window (0 = per-step form), row stride in records
  int box;           // windowed form: bytes of the stencil-box region at `tile` (0: none)
  int T[3];          // tile nodes per axis (all 0 = no tile)
  int tile_nodes;
};

// Tile box: every axis spans min(n, 2R + 1 + 2m) nodes for the largest margin
// m <= 24 that fits the byte budget; no tile if even m = 1 does not fit.
__host__ __device__ inline void tile_dims(const GridDev &g, const int *R, int budget, int *T) {
  T[0] = T[1] = T[2] = 0;
  if (budget <= 0) return;
  for (int m = 24; m >= 1; --m) {
    long long nodes = 1;
    int t[3] = {1, 1, 1};
    for (int k = 0; k < g.d; ++k) {
      int want = 2 * R[k] + 1 + 2 * m;
      t[k] = want < g.n[k] ? want : g.n[k];
      nodes *= t[k];
    }
    if (nodes * g.rec_bytes <= budget) {
      for (int k = 0; k < g.d; ++k) T[k] = t[k];
      return;
    }
  }
}

// window: the fused batched form, which runs eligible walkers windowed (and
// gives them no grid tile); mabp: the walker is an mABP walker.
__host__ __device__ inline GroupLayout group_layout(int natoms, const CvDev *cv, const GridDev &g, const int *R,
                                                    int nwarps, int rsz, int tile_budget, bool window = false,
                                                    bool mabp = false) {
  GroupLayout L;
  const int real = rsz / 4;
  int off = 0;
  L.win = window ? window_steps(natoms, cv, g.d, rsz) : 0;
  if (L.win) tile_budget = 0;
  L.xstride = natoms | 1;
  if (L.win) {
    const int rows = L.win * L.xstride * rsz;
    L.xs0 = off;
    off += rows;
    L.xs1 = off;
    off += rows;
    L.fs = L.xs0;
    L.steps = off;
    off += 3 * L.win * (rsz == 16 ? (int)sizeof(StepRec<float>) : (int)sizeof(StepRec<double>));
    off = align16(off);
    L.atoms = off;
    off += align16(natoms * 4) + natoms * kAtomTerms * (rsz == 16 ? 8 : 16);
  } else {
    L.xs0 = off;
    off += natoms * rsz;
    L.xs1 = off;
    off += natoms * rsz;
    L.fs = off;
    off += natoms * rsz;
    L.steps = L.atoms = off;
  }
  L.lists = off;
  for (int k = 0; k < g.d; ++k) {
    off += align16((cv[k].na + cv[k].nb) * 4);
    if (cv[k].type == ABP_CV_COM_DIST) off += align16((cv[k].na + cv[k].nb) * real);
  }
  off = align32(off);
  L.cn = off;
  for (int k = 0; k < g.d; ++k)
    if (cv[k].type == ABP_CV_COORD) off += (cv[k].na + cv[k].nb) * rsz + align32(nwarps * cv[k].na * 3 * real);
  off = align32(off);
  L.tile = off;
  L.box = 0;
  if (L.win) {
    for (int k = 0; k < 3; ++k) L.T[k] = 0;
    L.tile_nodes = 0;
    if (mabp) {
      L.box = kMabpBoxBytes;
    } else {
      // only a box the chain half can hold one node per thread of
      // (the window's single-round chain); larger boxes go round by round
      long long nodes = 1;
      for (int k = 0; k < g.d; ++k) nodes *= 2 * R[k] + 1;
      const int chain_threads = nwarps >= 2 ? nwarps * 16 : 32;
      if (g.d < 3 && nodes <= chain_threads && nodes * g.rec_bytes <= kWtBoxBytes)
        L.box = (int)(nodes * g.rec_bytes);
    }
    off += align16(L.box);
    L.total = align32(off);
    return L;
  }
  int budget = tile_budget - off;
  tile_dims(g, R, budget, L.T);
  L.tile_nodes = 0;
  if (L.T[0] > 0) {
    L.tile_nodes = 1;
    for (int k = 0; k < g.d; ++k) L.tile_nodes *= L.T[k];
    off += L.tile_nodes * g.rec_bytes;
  }
  L.total = align32(off);
  return L;
}

}  // namespace abp
