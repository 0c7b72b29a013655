// abp_device.cuh -- device building blocks of one walker step, executed by a
// "walker group" of G threads (one to eight warps) that owns the walker for
// the whole step. Every reduction runs in a fixed order, so a walker's result
// does not depend on which other walkers share the launch.
//
// Steps (arXiv:1609.09833):
//   a1 CVs + Jacobians          cv_com / cv_dihedral / cv_coord
//   a2 well-tempered height     interp_corners<double> + w exp(-V / dT)
//   a3 Gaussian stencil deposit build_tables + deposit_stencil
//   a4 multilinear interpolation interp_corners<Real>
//   a5 chain rule               scatter_forces
#pragma once

#include <math.h>

#include "abp_internal.cuh"

namespace abp {

// ---------------------------------------------------------------- records

struct __align__(32) D4 {
  double x, y, z, w;
};

template <typename Real>
struct Rec4;
template <>
struct Rec4<float> {
  using T = float4;
};
template <>
struct Rec4<double> {
  using T = D4;
};

template <typename Real>
__device__ __forceinline__ typename Rec4<Real>::T make_rec(Real x, Real y, Real z, Real w) {
  typename Rec4<Real>::T r;
  r.x = x;
  r.y = y;
  r.z = z;
  r.w = w;
  return r;
}

template <typename Real>
__device__ __forceinline__ typename Rec4<Real>::T ld_rec(const void *base, long long i) {
  return reinterpret_cast<const typename Rec4<Real>::T *>(base)[i];
}

// ---------------------------------------------------------------- groups

struct Grp {
  int G;       // threads in the group (multiple of 32)
  int gid;     // group index inside the CTA (named barrier gid + 1)
  int t;       // thread index inside the group
  int lane;
  int warp;    // warp index inside the group
  int nwarps;
  __device__ __forceinline__ void sync() const {
    if (G == 32) {
      __syncwarp();
    } else {
      __threadfence_block();
      asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(G) : "memory");
    }
  }
};

// Fixed per-group shared state.
template <typename Real>
struct GroupFixed {
  WalkerDev wd;
  Real red[kMaxGroupWarps * 8];
  double redd[kMaxGroupWarps * 8];
  double s[kMaxCv];           // CV values (FP32 arithmetic per term, FP64 sums)
  Real dvds[kMaxCv];
  Real com_u[kMaxCv][3];      // COM unit separation (J_A = -w u, J_B = +w u)
  Real dih_g[kMaxCv][4][3];   // dihedral gradient per atom
  double u[kMaxCv];           // fractional grid coordinate of s (deposit)
  int ic[kMaxCv];
  int ic_log[kMaxCv];         // floor(u + 1/2) before the out-of-range limit (deposit log)
  int flags;
  int bad;
  double V;                   // V_b(s_t) after the step's deposit (a4)
  double dV[kMaxCv];
  Real hf;                    // hill height (rounded to Real)
  Real tabG[kMaxCv][2 * kRMax + 1];
  Real tabD[kMaxCv][2 * kRMax + 1];
  int tabJ[kMaxCv][2 * kRMax + 1];
};

// Sum K values over the group; every thread receives the same total
// (lane-0 value of each warp, warps summed in index order).
template <int K, typename Real>
__device__ __forceinline__ void grp_sum(const Grp &g, Real (&v)[K], Real *red) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    v[k] = __shfl_sync(0xffffffffu, v[k], 0);
  }
  if (g.G == 32) return;
  if (g.lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) red[g.warp * 8 + k] = v[k];
  }
  g.sync();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    Real acc = 0;
    for (int w = 0; w < g.nwarps; ++w) acc += red[w * 8 + k];
    v[k] = acc;
  }
  g.sync();
}

template <typename Real>
__device__ __forceinline__ Real min_image(Real dx, double box, double inv_box) {
  return dx - (Real)box * floor(dx * (Real)inv_box + (Real)0.5);
}

template <typename Real>
__device__ __forceinline__ Real rcp_fast(Real x);
template <>
__device__ __forceinline__ float rcp_fast<float>(float x) {
  return __fdividef(1.0f, x);
}
template <>
__device__ __forceinline__ double rcp_fast<double>(double x) {
  return 1.0 / x;
}

// ---------------------------------------------------------------- a1: CVs

// Centre-of-mass distance s = |R_B - R_A| (minimum image if pbc). Each
// group's weighted sum runs over offsets from the group's first atom, which
// keeps the FP32 rounding at the scale of the group's extent rather than of
// the absolute coordinates: R_G = r_G + sum_i w_i (x_i - r_G), sum_i w_i = 1.
template <typename Real>
__device__ void cv_com(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs) {
  const CvDev &c = fx->wd.cv[k];
  const auto ra = xs[__ldg(c.ia)];
  const auto rb = xs[__ldg(c.ib)];
  Real v[6] = {0, 0, 0, 0, 0, 0};
  for (int i = g.t; i < c.na; i += g.G) {
    Real w = sizeof(Real) == 4 ? (Real)c.wa[i] : (Real)c.wa64[i];
    auto p = xs[__ldg(c.ia + i)];
    v[0] += w * (p.x - ra.x);
    v[1] += w * (p.y - ra.y);
    v[2] += w * (p.z - ra.z);
  }
  for (int i = g.t; i < c.nb; i += g.G) {
    Real w = sizeof(Real) == 4 ? (Real)c.wb[i] : (Real)c.wb64[i];
    auto p = xs[__ldg(c.ib + i)];
    v[3] += w * (p.x - rb.x);
    v[4] += w * (p.y - rb.y);
    v[5] += w * (p.z - rb.z);
  }
  grp_sum<6>(g, v, fx->red);
  if (g.t == 0) {
    Real d[3] = {(rb.x - ra.x) + (v[3] - v[0]), (rb.y - ra.y) + (v[4] - v[1]), (rb.z - ra.z) + (v[5] - v[2])};
    if (c.pbc)
      for (int q = 0; q < 3; ++q) d[q] = min_image(d[q], c.box[q], c.inv_box[q]);
    Real r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    fx->s[k] = (double)r;
    if (r > 0) {
      for (int q = 0; q < 3; ++q) fx->com_u[k][q] = d[q] / r;
    } else {
      for (int q = 0; q < 3; ++q) fx->com_u[k][q] = 0;
      fx->flags |= ABP_WFLAG_SINGULAR;
    }
  }
}

template <typename Real>
__device__ __forceinline__ void cross3(const Real *a, const Real *b, Real *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename Real>
__device__ __forceinline__ Real dot3(const Real *a, const Real *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Dihedral of atoms 1-2-3-4: phi = atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3)),
// gradient in the Blondel-Karplus form. One thread.
template <typename Real>
__device__ void cv_dihedral(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs) {
  if (g.t != 0) return;
  const CvDev &c = fx->wd.cv[k];
  Real x[4][3];
  for (int a = 0; a < 4; ++a) {
    auto p = xs[__ldg(c.ia + a)];
    x[a][0] = p.x;
    x[a][1] = p.y;
    x[a][2] = p.z;
  }
  Real b1[3], b2[3], b3[3], m[3], n[3];
  for (int q = 0; q < 3; ++q) {
    b1[q] = x[1][q] - x[0][q];
    b2[q] = x[2][q] - x[1][q];
    b3[q] = x[3][q] - x[2][q];
    if (c.pbc) {
      b1[q] = min_image(b1[q], c.box[q], c.inv_box[q]);
      b2[q] = min_image(b2[q], c.box[q], c.inv_box[q]);
      b3[q] = min_image(b3[q], c.box[q], c.inv_box[q]);
    }
  }
  cross3(b1, b2, m);
  cross3(b2, b3, n);
  Real lb2 = sqrt(dot3(b2, b2));
  fx->s[k] = (double)atan2(lb2 * dot3(b1, n), dot3(m, n));
  Real mm = dot3(m, m), nn = dot3(n, n);
  if (!(mm > 0) || !(nn > 0) || !(lb2 > 0)) {
    for (int a = 0; a < 4; ++a)
      for (int q = 0; q < 3; ++q) fx->dih_g[k][a][q] = 0;
    fx->flags |= ABP_WFLAG_SINGULAR;
    return;
  }
  Real inv_b2sq = 1 / (lb2 * lb2);
  Real p = dot3(b1, b2) * inv_b2sq, r = dot3(b3, b2) * inv_b2sq;
  for (int q = 0; q < 3; ++q) {
    Real g1 = -lb2 / mm * m[q];
    Real g4 = lb2 / nn * n[q];
    fx->dih_g[k][0][q] = g1;
    fx->dih_g[k][3][q] = g4;
    fx->dih_g[k][1][q] = -(1 + p) * g1 + r * g4;
    fx->dih_g[k][2][q] = -(1 + r) * g4 + p * g1;
  }
}

// Coordination number s = sum_{i in A, j in B} 1 / (1 + (r_ij / r0)^6)
// (the n = 6, m = 12 rational switch with the common factor cancelled).
// No square root: q = r^2 / r0^2, sw = 1 / (1 + q^3),
// d sw / d x_i = -6 q^2 sw^2 / r0^2 (x_i - x_j).
// Thread t owns B entries t, t + G, ... (JB per pass, gradients in registers);
// A entries are read from shared memory in chunks of 4 and their gradients
// are reduced over the warp, then summed over warps in a fixed order.
// jA / jB receive ds/dx per list entry.
template <typename Real>
__device__ void cv_coord(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs,
                         typename Rec4<Real>::T *jA, typename Rec4<Real>::T *jB, Real *lig) {
  using R4 = typename Rec4<Real>::T;
  const CvDev &c = fx->wd.cv[k];
  const Real k2 = (Real)c.inv_r0sq;
  const Real c6 = (Real)-6 * k2;
  const bool pbc = c.pbc != 0;
  const Real bx = (Real)c.box[0], by = (Real)c.box[1], bz = (Real)c.box[2];
  const Real ibx = (Real)c.inv_box[0], iby = (Real)c.inv_box[1], ibz = (Real)c.inv_box[2];
  Real *mylig = lig + g.warp * c.na * 3;
  for (int q = g.lane; q < c.na * 3; q += 32) mylig[q] = 0;
  __syncwarp();
  Real sacc = 0;  // this thread's partial sum (a few terms of size <= 1)
  constexpr int JB = 4;
  for (int jb0 = 0; jb0 < c.nb; jb0 += g.G * JB) {
    Real xj[JB], yj[JB], zj[JB], gxj[JB], gyj[JB], gzj[JB], mj[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      int j = jb0 + jj * g.G + g.t;
      bool ok = j < c.nb;
      R4 p = xs[__ldg(c.ib + (ok ? j : 0))];
      xj[jj] = p.x;
      yj[jj] = p.y;
      zj[jj] = p.z;
      mj[jj] = ok ? (Real)1 : (Real)0;
      gxj[jj] = gyj[jj] = gzj[jj] = 0;
    }
    for (int i0 = 0; i0 < c.na; i0 += 4) {
      Real gi[4][3];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        gi[ii][0] = gi[ii][1] = gi[ii][2] = 0;
        int i = i0 + ii;
        bool oki = i < c.na;
        R4 a = xs[__ldg(c.ia + (oki ? i : 0))];
#pragma unroll
        for (int jj = 0; jj < JB; ++jj) {
          Real dx = a.x - xj[jj], dy = a.y - yj[jj], dz = a.z - zj[jj];
          if (pbc) {
            dx = min_image(dx, bx, ibx);
            dy = min_image(dy, by, iby);
            dz = min_image(dz, bz, ibz);
          }
          Real q = (dx * dx + dy * dy + dz * dz) * k2;
          Real q2 = q * q;
          Real sw = rcp_fast<Real>((Real)1 + q2 * q);
          Real m = oki ? mj[jj] : (Real)0;
          sacc += m * sw;
          Real gf = c6 * m * q2 * sw * sw;
          gi[ii][0] += gf * dx;
          gi[ii][1] += gf * dy;
          gi[ii][2] += gf * dz;
          gxj[jj] -= gf * dx;
          gyj[jj] -= gf * dy;
          gzj[jj] -= gf * dz;
        }
      }
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          Real v = gi[ii][q];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (g.lane == 0 && i0 + ii < c.na) mylig[(i0 + ii) * 3 + q] += v;
        }
    }
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      int j = jb0 + jj * g.G + g.t;
      if (j < c.nb) jB[j] = make_rec<Real>(gxj[jj], gyj[jj], gzj[jj], (Real)0);
    }
  }
  // the sum of FP32 pair terms is reduced in FP64: a CN of a few hundred
  // needs more than FP32's 24 bits to place a hill two grid spacings wide
  double v[1] = {(double)sacc};
  grp_sum<1>(g, v, fx->redd);
  if (g.t == 0) fx->s[k] = v[0];
  g.sync();
  for (int i = g.t; i < c.na; i += g.G) {
    Real a0 = 0, a1 = 0, a2 = 0;
    for (int w = 0; w < g.nwarps; ++w) {
      const Real *L = lig + w * c.na * 3 + i * 3;
      a0 += L[0];
      a1 += L[1];
      a2 += L[2];
    }
    jA[i] = make_rec<Real>(a0, a1, a2, (Real)0);
  }
}

// ---------------------------------------------------------------- grid helpers

// Fractional coordinate of s along axis k; periodic axes wrapped into [0, n).
// (Any finite or non-finite s maps to a u whose stencil indices stay in
// range: a periodic u is forced into [0, n); a non-periodic u far outside the
// axis is limited so that its box holds no node.)
__device__ __forceinline__ double axis_u(const GridDev &gd, int k, double s, int R) {
  double u = (s - gd.lo[k]) * gd.invD[k];
  double n = (double)gd.n[k];
  if (gd.periodic[k]) {
    u = u - n * floor(u / n);
    if (u >= n) u -= n;
    if (u < 0) u += n;
    if (!(u >= 0.0 && u < n)) u = 0.0;
  } else {
    if (!(u >= -R - 2.0)) u = -R - 2.0;
    if (!(u <= n + R + 1.0)) u = n + R + 1.0;
  }
  return u;
}

// Load node `node` of the grid as 1 + d values (value + compensation).
template <typename Acc>
__device__ __forceinline__ void load_node(const GridDev &gd, long long node, Acc *v) {
  if (gd.prec == ABP_PREC_FP32_COMP) {
    if (gd.d == 1) {
      float4 r = reinterpret_cast<const float4 *>(gd.rec)[node];
      v[0] = (Acc)r.x + (Acc)r.z;
      v[1] = (Acc)r.y + (Acc)r.w;
    } else {
      const float4 *p = reinterpret_cast<const float4 *>(gd.rec) + 2 * node;
      float4 a = p[0], b = p[1];
      v[0] = (Acc)a.x + (Acc)b.x;
      v[1] = (Acc)a.y + (Acc)b.y;
      v[2] = (Acc)a.z + (Acc)b.z;
      v[3] = (Acc)a.w + (Acc)b.w;
    }
  } else {
    if (gd.d == 1) {
      const double2 r = reinterpret_cast<const double2 *>(gd.rec)[node];
      v[0] = (Acc)r.x;
      v[1] = (Acc)r.y;
    } else {
      const D4 r = reinterpret_cast<const D4 *>(gd.rec)[node];
      v[0] = (Acc)r.x;
      v[1] = (Acc)r.y;
      v[2] = (Acc)r.z;
      v[3] = (Acc)r.w;
    }
  }
}

// a4: multilinear interpolation of V and dV/dxi_k at s, by the first 2^d
// lanes of warp 0 of the group (one corner per lane), combined with a fixed
// xor-butterfly. Non-periodic axes clamp s to the range and report a zero
// gradient along a clamped axis. Result valid in lane 0 of warp 0.
template <typename Acc>
__device__ __forceinline__ int interp_corners(const GridDev &gd, const double *s, int lane, Acc *out) {
  int d = gd.d;
  int i0[3] = {0, 0, 0}, i1[3] = {0, 0, 0}, clamped = 0;
  Acc f[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    double u = (s[k] - gd.lo[k]) * gd.invD[k];
    int n = gd.n[k];
    if (gd.periodic[k]) {
      u = u - (double)n * floor(u / (double)n);
      if (u >= (double)n) u -= (double)n;
      if (u < 0) u += (double)n;
      if (!(u >= 0.0 && u < (double)n)) u = 0.0;
      int a = (int)floor(u);
      if (a > n - 1) a = n - 1;
      i0[k] = a;
      i1[k] = (a + 1 == n) ? 0 : a + 1;
      f[k] = (Acc)(u - (double)a);
    } else {
      if (!(u >= 0)) {
        u = 0;
        clamped |= 1 << k;
      }
      if (u > (double)(n - 1)) {
        u = (double)(n - 1);
        clamped |= 1 << k;
      }
      int a = (int)floor(u);
      if (a > n - 2) a = n - 2;
      i0[k] = a;
      i1[k] = a + 1;
      f[k] = (Acc)(u - (double)a);
    }
  }
  Acc acc[4] = {0, 0, 0, 0};
  if (lane < (1 << d)) {
    Acc wgt = 1;
    long long node = 0, mul = 1;
    for (int k = 0; k < d; ++k) {
      int hi = (lane >> k) & 1;
      wgt *= hi ? f[k] : (Acc)1 - f[k];
      node += mul * (hi ? i1[k] : i0[k]);
      mul *= gd.n[k];
    }
    Acc v[4];
    load_node<Acc>(gd, node, v);
    for (int q = 0; q <= d; ++q) acc[q] = wgt * v[q];
  }
  for (int q = 0; q < 4; ++q)
    for (int o = 1; o < 8; o <<= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  out[0] = acc[0];
  for (int k = 0; k < d; ++k) out[1 + k] = (clamped >> k) & 1 ? (Acc)0 : acc[1 + k];
  return clamped ? ABP_WFLAG_OOR : 0;
}

// a3 (part 1): per-axis factor tables of the stencil box around s:
// node index j (or -1 outside a non-periodic axis), G_k = exp(-d^2 / 2 sigma^2)
// and -d / sigma^2, d = (j_unwrapped - u) D the node-to-centre distance.
template <typename Real>
__device__ void build_tables(const Grp &g, GroupFixed<Real> *fx) {
  const WalkerDev &wd = fx->wd;
  const GridDev &gd = wd.g;
  if (g.t < gd.d) {
    int k = g.t;
    double u = axis_u(gd, k, fx->s[k], fx->wd.R[k]);
    int ic = (int)floor(u + 0.5);
    if (!gd.periodic[k]) {
      double raw = (fx->s[k] - gd.lo[k]) * gd.invD[k] + 0.5;
      raw = raw > 1e9 ? 1e9 : (raw < -1e9 ? -1e9 : raw);
      fx->ic_log[k] = (int)floor(raw == raw ? raw : 0.0);
    }
    if (gd.periodic[k] && ic >= gd.n[k]) {
      // u in [n - 1/2, n): the nearest node is node 0, one period up
      ic -= gd.n[k];
      u -= gd.n[k];
    }
    fx->u[k] = u;
    fx->ic[k] = ic;
    if (gd.periodic[k]) fx->ic_log[k] = ic;
  }
  g.sync();
  for (int k = 0; k < gd.d; ++k) {
    int R = wd.R[k], span = 2 * R + 1, n = gd.n[k];
    double u = fx->u[k];
    int ic = fx->ic[k];
    Real i2 = (Real)wd.inv2s2[k], is2 = (Real)wd.invs2[k];
    for (int o = g.t; o < span; o += g.G) {
      int j = ic - R + o;
      Real dist = (Real)(((double)j - u) * gd.D[k]);
      int jj = j;
      if (gd.periodic[k]) {
        jj = j % n;
        if (jj < 0) jj += n;
      } else if (j < 0 || j >= n) {
        jj = -1;
      }
      fx->tabJ[k][o] = jj;
      fx->tabG[k][o] = exp(-dist * dist * i2);
      fx->tabD[k][o] = -dist * is2;
    }
  }
}

__device__ __forceinline__ void two_sum_add(float &s, float &c, float x) {
  float t = __fadd_rn(s, x);
  float bp = __fsub_rn(t, s);
  float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
  s = t;
  c = __fadd_rn(c, e);
}

// a3 (part 2): add h G and h G (-d_k / sigma_k^2) at every in-range node of
// the box. FP32_COMP grids accumulate with two-sum compensation; FP64 grids
// add directly. Each walker's grid has a single writer (its group).
template <typename Real>
__device__ void deposit_stencil(const Grp &g, GroupFixed<Real> *fx) {
  const WalkerDev &wd = fx->wd;
  const GridDev &gd = wd.g;
  const int d = gd.d;
  const int s0 = 2 * wd.R[0] + 1;
  const int s1 = d > 1 ? 2 * wd.R[1] + 1 : 1;
  const int s2 = d > 2 ? 2 * wd.R[2] + 1 : 1;
  const int total = s0 * s1 * s2;
  const Real h = fx->hf;
  const long long n0 = gd.n[0], n01 = (long long)gd.n[0] * (d > 1 ? gd.n[1] : 1);
  for (int idx = g.t; idx < total; idx += g.G) {
    int o0 = idx % s0;
    int r = idx / s0;
    int o1 = r % s1;
    int o2 = r / s1;
    int j0 = fx->tabJ[0][o0];
    int j1 = d > 1 ? fx->tabJ[1][o1] : 0;
    int j2 = d > 2 ? fx->tabJ[2][o2] : 0;
    if ((j0 | j1 | j2) < 0) continue;
    Real G = h * fx->tabG[0][o0];
    if (d > 1) G = G * fx->tabG[1][o1];
    if (d > 2) G = G * fx->tabG[2][o2];
    long long node = j0 + n0 * j1 + n01 * j2;
    if constexpr (sizeof(Real) == 4) {
      if (d == 1) {
        float4 *p = reinterpret_cast<float4 *>(gd.rec) + node;
        float4 v = *p;
        two_sum_add(v.x, v.z, G);
        two_sum_add(v.y, v.w, __fmul_rn(G, fx->tabD[0][o0]));
        *p = v;
      } else {
        float4 *p = reinterpret_cast<float4 *>(gd.rec) + 2 * node;
        float4 a = p[0], b = p[1];
        two_sum_add(a.x, b.x, G);
        two_sum_add(a.y, b.y, __fmul_rn(G, fx->tabD[0][o0]));
        two_sum_add(a.z, b.z, __fmul_rn(G, fx->tabD[1][o1]));
        if (d > 2) two_sum_add(a.w, b.w, __fmul_rn(G, fx->tabD[2][o2]));
        p[0] = a;
        p[1] = b;
      }
    } else {
      if (d == 1) {
        double2 *p = reinterpret_cast<double2 *>(gd.rec) + node;
        double2 v = *p;
        v.x += G;
        v.y += G * fx->tabD[0][o0];
        *p = v;
      } else {
        D4 *p = reinterpret_cast<D4 *>(gd.rec) + node;
        D4 v = *p;
        v.x += G;
        v.y += G * fx->tabD[0][o0];
        v.z += G * fx->tabD[1][o1];
        if (d > 2) v.w += G * fx->tabD[2][o2];
        *p = v;
      }
    }
  }
}

// ---------------------------------------------------------------- a5

// F_i = - sum_k dV/ds_k ds_k/dx_i into the force accumulators fs (zeroed by
// the caller). Lists are unique, and each list is a separate phase, so every
// accumulator is updated in a fixed order.
template <typename Real>
__device__ void scatter_forces(const Grp &g, GroupFixed<Real> *fx, typename Rec4<Real>::T *fs,
                               unsigned char *cnmem) {
  using R4 = typename Rec4<Real>::T;
  const WalkerDev &wd = fx->wd;
  int d = wd.g.d;
  int rsz = (int)sizeof(R4);
  unsigned char *cur = cnmem;
  for (int k = 0; k < d; ++k) {
    const CvDev &c = wd.cv[k];
    Real dv = fx->dvds[k];
    if (c.type == ABP_CV_COM_DIST) {
      Real ux = fx->com_u[k][0] * dv, uy = fx->com_u[k][1] * dv, uz = fx->com_u[k][2] * dv;
      for (int i = g.t; i < c.na; i += g.G) {
        Real w = sizeof(Real) == 4 ? (Real)c.wa[i] : (Real)c.wa64[i];
        R4 &f = fs[__ldg(c.ia + i)];
        f.x += w * ux;
        f.y += w * uy;
        f.z += w * uz;
      }
      g.sync();
      for (int i = g.t; i < c.nb; i += g.G) {
        Real w = sizeof(Real) == 4 ? (Real)c.wb[i] : (Real)c.wb64[i];
        R4 &f = fs[__ldg(c.ib + i)];
        f.x -= w * ux;
        f.y -= w * uy;
        f.z -= w * uz;
      }
      g.sync();
    } else if (c.type == ABP_CV_DIHEDRAL) {
      if (g.t < 4) {
        R4 &f = fs[__ldg(c.ia + g.t)];
        f.x -= dv * fx->dih_g[k][g.t][0];
        f.y -= dv * fx->dih_g[k][g.t][1];
        f.z -= dv * fx->dih_g[k][g.t][2];
      }
      g.sync();
    } else {
      const R4 *jA = reinterpret_cast<const R4 *>(cur);
      const R4 *jB = jA + c.na;
      for (int i = g.t; i < c.na; i += g.G) {
        R4 &f = fs[__ldg(c.ia + i)];
        R4 j = jA[i];
        f.x -= dv * j.x;
        f.y -= dv * j.y;
        f.z -= dv * j.z;
      }
      g.sync();
      for (int i = g.t; i < c.nb; i += g.G) {
        R4 &f = fs[__ldg(c.ib + i)];
        R4 j = jB[i];
        f.x -= dv * j.x;
        f.y -= dv * j.y;
        f.z -= dv * j.z;
      }
      g.sync();
      int lig = (g.nwarps * c.na * 3 * (int)sizeof(Real) + 31) & ~31;
      cur += (c.na + c.nb) * rsz + lig;
    }
  }
}

}  // namespace abp
