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
  int pbc;
  double box[3];
  double inv_box[3];
};

struct GridDev {
  int d;
  int n[3];
  int periodic[3];
  double lo[3];
  double D[3];       // node spacing
  double invD[3];
  double L[3];       // axis length (periodic wrap)
  int prec;          // ABP_PREC_*
  int rec_bytes;     // bytes per node record
  long long nodes;
  void *rec;         // node records (see GridLayout below)
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
  void *fbuf;        // library-owned force records (abp_step -> abp_forces)
  void *jscratch;    // library-owned Jacobian scratch (plain form)
  WalkerState *state;
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
  int pad[31];
};

// Bytes of dynamic shared memory one walker group needs beyond its fixed
// part, for a walker with these CVs (computed identically on host and
// device). rsz = bytes of one 4-component record (16 for float, 32 double).
__host__ __device__ inline int group_dyn_bytes(int natoms, const CvDev *cv, int ncv, int nwarps, int rsz) {
  int b = 2 * natoms * rsz;  // coordinates + force accumulators
  int real = rsz / 4;
  for (int k = 0; k < ncv; ++k) {
    if (cv[k].type == ABP_CV_COORD) {
      b += (cv[k].na + cv[k].nb) * rsz;                       // dCN/dx per list entry
      int lig = nwarps * cv[k].na * 3 * real;                 // per-warp ligand partials
      b += (lig + 31) & ~31;
    }
  }
  return b;
}

}  // namespace abp
