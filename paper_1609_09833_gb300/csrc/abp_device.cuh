// abp_device.cuh -- device building blocks of one walker step, executed by a
// "walker group" of G threads (one to eight warps) that owns the walker for
// all steps of a launch. Every reduction runs in a fixed order, so a walker's
// result does not depend on which other walkers share the launch, and the
// optional shared-memory grid tile is an exact cache of the grid (same values,
// same arithmetic), so it does not change results either.
//
// Steps (arXiv:1609.09833):
//   a1 CVs + Jacobians           cv_com / cv_dihedral / cv_coord
//   a2 well-tempered height      height_interp + w exp(-V / dT)
//   a3 Gaussian stencil deposit  build_tables + deposit_stencil
//   a4 multilinear interpolation interp_step
//   a5 chain rule                scatter_forces
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

// 16-byte asynchronous global -> shared copy (completes at cp_async_wait).
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
// The same with an L2 eviction-priority policy (see l2_evict_first).
__device__ __forceinline__ void cp_async16_hint(void *smem_dst, const void *gmem_src, unsigned long long policy) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem_src), "l"(policy)
               : "memory");
}
// L2 policy for data read once (streamed coordinates): evicted first, so the
// grids that are read and written again keep their lines.
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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
  Real sh[kMaxCv], sl[kMaxCv];  // CV value s = sh + sl (sl carries the low bits of long FP32 sums)
  Real dvds[kMaxCv];
  Real com_u[kMaxCv][3];     // COM unit separation (J_A = -w u, J_B = +w u)
  Real dih_g[kMaxCv][4][3];  // dihedral gradient per atom
  // per-step axis state (one thread per axis)
  int i0[kMaxCv], i1[kMaxCv];  // interpolation corners
  Real f[kMaxCv];            // interpolation weight of i1
  int da[kMaxCv];            // deposit: node below u (unwrapped)
  Real df[kMaxCv];           // deposit: u - da, in [0, 1)
  int dc[kMaxCv];            // deposit: centre offset, i_c = da + dc (dc = 1 iff df >= 1/2)
  int ic_log[kMaxCv];        // i_c for the deposit log (wrapped; unclamped outside a range)
  int clamped;               // interpolation clamp mask
  int flags;
  int bad;
  unsigned winbad[3];        // windowed form: non-finite steps of the windows in flight (window % 3)
  int reload;                // the tile must be reloaded this step
  int org[kMaxCv];           // tile origin node per axis
  Real V;
  Real dV[kMaxCv];
  Real hf;                   // hill height (rounded to Real)
  double hV;                 // windowed form: V_b(s_t) before the deposit at hand
  // atom lists of each CV (shared memory, or global in the plain form)
  const int32_t *ia[kMaxCv];
  const int32_t *ib[kMaxCv];
  const Real *wa[kMaxCv];
  const Real *wb[kMaxCv];
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

// Any thread of the group set `flag`?
template <typename Real>
__device__ __forceinline__ bool grp_any(const Grp &g, GroupFixed<Real> *fx, int flag) {
  int w = __any_sync(0xffffffffu, flag);
  if (g.G == 32) return w != 0;
  if (g.t == 0) fx->bad = 0;
  g.sync();
  if (g.lane == 0 && w) fx->bad = 1;
  g.sync();
  int r = fx->bad;
  g.sync();
  return r != 0;
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

// Error-free sum a + b = s + e (two-sum); exact in round-to-nearest.
// A grid node index about to be read or written. The checked build
// (compiled with -DABP_CHECKED, the substitute for a memory checker) counts
// an index outside [0, nodes) in the context's counters and returns node 0,
// so that the access stays inside the grid; the normal build returns the
// index unchanged.
__device__ __forceinline__ long long chk_node(const GridDev &gd, long long node) {
#ifdef ABP_CHECKED
  if (node < 0 || node >= gd.nodes) {
    if (gd.oob) atomicAdd(gd.oob, 1ull);
    return 0;
  }
#endif
  return node;
}

template <typename Real>
__device__ __forceinline__ void two_sum(Real a, Real b, Real &s, Real &e);
template <>
__device__ __forceinline__ void two_sum<float>(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
template <>
__device__ __forceinline__ void two_sum<double>(double a, double b, double &s, double &e) {
  s = __dadd_rn(a, b);
  double bp = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bp)), __dsub_rn(b, bp));
}

// (ah, al) += (bh, bl) in hi + lo ("double-single") arithmetic, renormalized.
// Commutative bit for bit, since two_sum's error term is exact.
template <typename Real>
__device__ __forceinline__ void ff_add(Real &ah, Real &al, Real bh, Real bl) {
  Real s, e;
  two_sum<Real>(ah, bh, s, e);
  e = e + (al + bl);
  ah = s + e;
  al = e - (ah - s);
}

// Group sum of a hi + lo pair (fixed order, all threads get the total).
template <typename Real>
__device__ __forceinline__ void grp_sum_ff(const Grp &g, Real &h, Real &l, Real *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Real oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    ff_add<Real>(h, l, oh, ol);
  }
  h = __shfl_sync(0xffffffffu, h, 0);
  l = __shfl_sync(0xffffffffu, l, 0);
  if (g.G == 32) return;
  if (g.lane == 0) {
    red[g.warp * 8] = h;
    red[g.warp * 8 + 1] = l;
  }
  g.sync();
  h = red[0];
  l = red[1];
  for (int w = 1; w < g.nwarps; ++w) ff_add<Real>(h, l, red[w * 8], red[w * 8 + 1]);
  g.sync();
}

// ---------------------------------------------------------------- a1: CVs

// The end of an FP32 COM distance in hi + lo arithmetic: d = (r_B - r_A) +
// (B - A), r_G each group's first atom and G + Gl its weighted offset sum
// (hi + lo, not necessarily normalised), the first atoms' difference and the
// sums' difference formed exactly; a minimum image in a periodic box;
// r^2 = sum d^2 as an FP32 sum S of the squares' high parts plus their
// exact errors and low terms (Ogita, Rump and Oishi's Sum2 kept unrounded),
// and s = sh + sl from an approximate root sh = S / sqrt(S) corrected by one
// Newton step on the residual S + r2l - sh^2 (exact by fma); u = d / s in
// FP32. A hill two grid spacings wide on a fine grid needs s to ~1e-6 of its
// width, below the resolution of one FP32 number near 1 nm. The chain is
// kept short (each value's low part rides beside it unnormalised): it is
// the longest dependency of a COM-distance step.
__device__ __forceinline__ int com_finish_ff(const CvDev &c, const float *ra, const float *ah, const float *al,
                                             const float *rb, const float *bh, const float *bl, float &sh, float &sl,
                                             float *u) {
  float dh[3], dl[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float rdh, rdl, t, te, s1, e1;
    float gah = ah[q], gal = al[q], gbh = bh[q], gbl = bl[q];
    // equal masses: the weights' FP32 rounding, one factor per group
    if (c.wc_a != 0.f) ff_add<float>(gah, gal, __fmul_rn(gah, c.wc_a), 0.f);
    if (c.wc_b != 0.f) ff_add<float>(gbh, gbl, __fmul_rn(gbh, c.wc_b), 0.f);
    two_sum<float>(rb[q], -ra[q], rdh, rdl);
    two_sum<float>(gbh, -gah, t, te);
    two_sum<float>(rdh, t, s1, e1);
    // every low term is far below s1 unless d itself is (a coincidence of
    // the two centres, where the direction u carries no information)
    dh[q] = s1;
    dl[q] = __fadd_rn(__fadd_rn(e1, te), __fadd_rn(rdl, __fsub_rn(gbl, gal)));
    if (c.pbc) {
      const float n = __fadd_rn(dh[q], dl[q]);
      dl[q] = __fsub_rn(dl[q], __fsub_rn(n, dh[q]));
      dh[q] = n;
      const float shift = __fmul_rn((float)c.box[q], floorf(__fmaf_rn(dh[q], (float)c.inv_box[q], 0.5f)));
      float t2, te2;
      two_sum<float>(dh[q], -shift, t2, te2);
      dh[q] = t2;
      dl[q] = __fadd_rn(dl[q], te2);
    }
  }
  float p[3], e[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    p[q] = __fmul_rn(dh[q], dh[q]);
    e[q] = __fmaf_rn(__fmul_rn(2.f, dh[q]), dl[q], __fmaf_rn(dh[q], dh[q], -p[q]));
  }
  float S1, c1, S, c2;
  two_sum<float>(p[0], p[1], S1, c1);
  two_sum<float>(S1, p[2], S, c2);
  const float r2l = __fadd_rn(__fadd_rn(c1, c2), __fadd_rn(__fadd_rn(e[0], e[1]), e[2]));
  if (S > 0.f) {
    // ir ~ 1 / sqrt(S) to a few units in the last place; the Newton step
    // makes sh + sl the root of S + r2l to ~2^-44 whatever sh's last bits,
    // and u only needs FP32 accuracy
    const float ir = rsqrtf(S);
    const float rh = __fmul_rn(S, ir);
    sh = rh;
    sl = __fmul_rn(__fadd_rn(__fmaf_rn(-rh, rh, S), r2l), __fmul_rn(0.5f, ir));
#pragma unroll
    for (int q = 0; q < 3; ++q) u[q] = __fmul_rn(dh[q], ir);
    return 0;
  }
  sh = S == S ? 0.f : S;  // coincident centres: 0; non-finite coordinates: NaN
  sl = 0.f;
#pragma unroll
  for (int q = 0; q < 3; ++q) u[q] = 0.f;
  return ABP_WFLAG_SINGULAR;
}

// Centre-of-mass distance s = |R_B - R_A| (minimum image if pbc). Each
// group's weighted sum runs over offsets from the group's first atom, which
// keeps the rounding at the scale of the group's extent rather than of the
// absolute coordinates: R_G = r_G + sum_i w_i (x_i - r_G), sum_i w_i = 1.
// FP32 walkers sum every weighted offset exactly as hi + lo (the difference
// x - r_G split by two_sum, the product's error by fma; the tiny w times the
// difference's low part rounded once) with two_sum per thread and hi + lo
// across the group, and finish in hi + lo (com_finish_ff): a group of
// hundreds of atoms spread over nanometres would otherwise lose ~1e-7 nm,
// several millionths of a hill a few grid spacings wide.
template <typename Real>
__device__ void cv_com(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs) {
  const CvDev &c = fx->wd.cv[k];
  const int32_t *ia = fx->ia[k], *ib = fx->ib[k];
  const Real *wa = fx->wa[k], *wb = fx->wb[k];
  const auto ra = xs[ia[0]];
  const auto rb = xs[ib[0]];
  if constexpr (sizeof(Real) == 4) {
    float h[6] = {0, 0, 0, 0, 0, 0}, l[6] = {0, 0, 0, 0, 0, 0};
    auto acc = [&](int q, float w, float x, float r) {
      float dh, dl;
      two_sum<float>(x, -r, dh, dl);  // x - r exactly
      const float ph = __fmul_rn(w, dh);
      const float pl = __fmaf_rn(w, dl, __fmaf_rn(w, dh, -ph));
      float t, e;
      two_sum<float>(h[q], ph, t, e);
      h[q] = t;
      l[q] = __fadd_rn(l[q], __fadd_rn(e, pl));
    };
    for (int i = g.t; i < c.na; i += g.G) {
      const float w = wa[i];
      const auto p = xs[ia[i]];
      acc(0, w, p.x, ra.x);
      acc(1, w, p.y, ra.y);
      acc(2, w, p.z, ra.z);
    }
    for (int i = g.t; i < c.nb; i += g.G) {
      const float w = wb[i];
      const auto p = xs[ib[i]];
      acc(3, w, p.x, rb.x);
      acc(4, w, p.y, rb.y);
      acc(5, w, p.z, rb.z);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      // the running sum and its low part as a normalised hi + lo pair
      float s2, e2;
      two_sum<float>(h[q], l[q], s2, e2);
      h[q] = s2;
      l[q] = e2;
      grp_sum_ff<float>(g, h[q], l[q], fx->red);
    }
    if (g.t == 0) {
      const float r0a[3] = {ra.x, ra.y, ra.z}, r0b[3] = {rb.x, rb.y, rb.z};
      float sh, sl;
      const int fl = com_finish_ff(c, r0a, h, l, r0b, h + 3, l + 3, sh, sl, fx->com_u[k]);
      fx->sh[k] = sh;
      fx->sl[k] = sl;
      if (fl) fx->flags |= fl;
    }
    return;
  }
  Real v[6] = {0, 0, 0, 0, 0, 0};
  for (int i = g.t; i < c.na; i += g.G) {
    Real w = wa[i];
    auto p = xs[ia[i]];
    v[0] += w * (p.x - ra.x);
    v[1] += w * (p.y - ra.y);
    v[2] += w * (p.z - ra.z);
  }
  for (int i = g.t; i < c.nb; i += g.G) {
    Real w = wb[i];
    auto p = xs[ib[i]];
    v[3] += w * (p.x - rb.x);
    v[4] += w * (p.y - rb.y);
    v[5] += w * (p.z - rb.z);
  }
  grp_sum<6>(g, v, fx->red);
  if (g.t == 0) {
    Real d[3] = {(rb.x - ra.x) + (v[3] - v[0]), (rb.y - ra.y) + (v[4] - v[1]), (rb.z - ra.z) + (v[5] - v[2])};
    if (c.pbc)
      for (int q = 0; q < 3; ++q) d[q] = min_image(d[q], c.box[q], c.inv_box[q]);
    Real r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    Real r = sqrt(r2);
    fx->sh[k] = r;
    fx->sl[k] = 0;
    if (r > 0) {
      Real ir = rcp_fast<Real>(r);
      for (int q = 0; q < 3; ++q) fx->com_u[k][q] = d[q] * ir;
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

// The dihedral angle of FP32 coordinates formed in FP64 (the coordinates
// and their differences are exact there): for hills so narrow that the FP32
// angle's rounding, ~1e-7 rad near +-pi, would move them by more than a few
// millionths of their width.
__device__ __forceinline__ double dihedral_angle64(const CvDev &c, const float (&x)[4][3]) {
  double b1[3], b2[3], b3[3], m[3], n[3];
  for (int q = 0; q < 3; ++q) {
    b1[q] = (double)x[1][q] - (double)x[0][q];
    b2[q] = (double)x[2][q] - (double)x[1][q];
    b3[q] = (double)x[3][q] - (double)x[2][q];
    if (c.pbc) {
      b1[q] = min_image<double>(b1[q], c.box[q], c.inv_box[q]);
      b2[q] = min_image<double>(b2[q], c.box[q], c.inv_box[q]);
      b3[q] = min_image<double>(b3[q], c.box[q], c.inv_box[q]);
    }
  }
  cross3<double>(b1, b2, m);
  cross3<double>(b2, b3, n);
  return atan2(sqrt(dot3<double>(b2, b2)) * dot3<double>(b1, n), dot3<double>(m, n));
}

// Dihedral of atoms 1-2-3-4 at positions x: phi = atan2(|b2| b1.(b2 x b3),
// (b1 x b2).(b2 x b3)), gradient in the Blondel-Karplus form, by one thread.
// phi_lo receives the low part of the angle: 0, or with c.hp (FP32 walkers)
// the FP64 angle's remainder after its FP32 rounding phi.
template <typename Real>
__device__ __forceinline__ int dihedral_core(const CvDev &c, const Real (&x)[4][3], Real &phi, Real (*grad)[3],
                                             Real &phi_lo) {
  phi_lo = 0;
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
  Real b2sq = dot3(b2, b2);
  Real lb2 = sqrt(b2sq);
  if constexpr (sizeof(Real) == 4) {
    if (c.hp) {
      const double p64 = dihedral_angle64(c, x);
      phi = (float)p64;
      phi_lo = (float)(p64 - (double)phi);
    } else {
      phi = atan2(lb2 * dot3(b1, n), dot3(m, n));
    }
  } else {
    phi = atan2(lb2 * dot3(b1, n), dot3(m, n));
  }
  Real mm = dot3(m, m), nn = dot3(n, n);
  if (!(mm > 0) || !(nn > 0) || !(lb2 > 0)) {
    for (int a = 0; a < 4; ++a)
      for (int q = 0; q < 3; ++q) grad[a][q] = 0;
    return ABP_WFLAG_SINGULAR;
  }
  Real inv_b2sq = rcp_fast<Real>(b2sq);
  Real p = dot3(b1, b2) * inv_b2sq, r = dot3(b3, b2) * inv_b2sq;
  Real cm = -lb2 * rcp_fast<Real>(mm), cn = lb2 * rcp_fast<Real>(nn);
  for (int q = 0; q < 3; ++q) {
    Real g1 = cm * m[q];
    Real g4 = cn * n[q];
    grad[0][q] = g1;
    grad[3][q] = g4;
    grad[1][q] = -(1 + p) * g1 + r * g4;
    grad[2][q] = -(1 + r) * g4 + p * g1;
  }
  return 0;
}

// The dihedral of the atoms ia[0..3] of xs (dihedral_core).
template <typename Real>
__device__ __forceinline__ int dihedral_eval(const CvDev &c, const int32_t *ia, const typename Rec4<Real>::T *xs,
                                             Real &phi, Real (*grad)[3], Real &phi_lo) {
  Real x[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    auto p = xs[ia[a]];
    x[a][0] = p.x;
    x[a][1] = p.y;
    x[a][2] = p.z;
  }
  return dihedral_core<Real>(c, x, phi, grad, phi_lo);
}

template <typename Real>
__device__ void cv_dihedral(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs) {
  if (g.t != g.G - 1) return;
  Real phi, phi_lo;
  int fl = dihedral_eval<Real>(fx->wd.cv[k], fx->ia[k], xs, phi, fx->dih_g[k], phi_lo);
  fx->sh[k] = phi;
  fx->sl[k] = phi_lo;
  if (fl) fx->flags |= fl;
}

// Coordination number s = sum_{i in A, j in B} 1 / (1 + (r_ij / r0)^6)
// (the n = 6, m = 12 rational switch with the common factor cancelled).
// No square root: q = r^2 / r0^2, sw = 1 / (1 + q^3),
// d sw / d x_i = -6 q^2 sw^2 / r0^2 (x_i - x_j).
// Thread t owns B entries t, t + G, ... (JB per pass, gradients in registers);
// A entries are read from shared memory in chunks of 4 and their gradients
// are reduced over the warp, then summed over warps in a fixed order.
// jA / jB receive ds/dx per list entry.
// Coordination number for a group A of at most 4 * MAXA atoms, tiled over
// the group's threads: lane & 3 picks one of four A-groups (A atoms i with
// i % 4 == lane & 3, held in registers with their gradients) and t >> 2 one
// of G/4 B-groups (B atoms j with j % (G/4) == t >> 2, streamed). Every pair
// is evaluated once. A B atom's gradient is summed over its four A-groups by
// two lane exchanges; A gradients over the B-groups once, at the end (lane
// exchanges, then warps in index order). Four compensated chains per thread.
template <typename Real, int MAXA>
__device__ void cv_coord_tiled(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs,
                               typename Rec4<Real>::T *jA, typename Rec4<Real>::T *jB, Real *lig) {
  using R4 = typename Rec4<Real>::T;
  const CvDev &c = fx->wd.cv[k];
  const int32_t *ia = fx->ia[k], *ib = fx->ib[k];
  const Real k2 = (Real)c.inv_r0sq;
  const Real c6 = (Real)-6 * k2;
  const bool pbc = c.pbc != 0;
  const Real bx = (Real)c.box[0], by = (Real)c.box[1], bz = (Real)c.box[2];
  const Real ibx = (Real)c.inv_box[0], iby = (Real)c.inv_box[1], ibz = (Real)c.inv_box[2];
  const int ag = g.lane & 3, bgrp = g.t >> 2, nbg = g.G >> 2;
  Real ax[MAXA], ay[MAXA], az[MAXA], gx[MAXA], gy[MAXA], gz[MAXA];
#pragma unroll
  for (int q = 0; q < MAXA; ++q) {
    const int i = ag + 4 * q;
    gx[q] = gy[q] = gz[q] = 0;
    ax[q] = ay[q] = az[q] = 0;
    if (i < c.na) {
      const R4 p = xs[ia[i]];
      ax[q] = p.x;
      ay[q] = p.y;
      az[q] = p.z;
    }
  }
  // s: each B round's switch values summed in A order, the round's sum then
  // added to a compensated (two-sum) accumulator
  Real sacc = 0, scomp = 0;
  // rows of A atoms this lane holds (the last row may be short)
  const int nrow = (c.na - ag + 3) >> 2;
  // every lane runs the same number of B rounds (the lane exchanges need the
  // whole warp); in the last round a lane past the end of B skips the pairs
  const int rounds = (c.nb + nbg - 1) / nbg;
  for (int rj = 0; rj < rounds; ++rj) {
    const int j = bgrp + rj * nbg;
    const bool okj = j < c.nb;
    Real gjx = 0, gjy = 0, gjz = 0;
    if (okj) {
      const R4 p = xs[ib[j]];
      Real part = 0;
#pragma unroll
      for (int q = 0; q < MAXA; ++q) {
        if (q < nrow) {
          Real dx = ax[q] - p.x, dy = ay[q] - p.y, dz = az[q] - p.z;
          if (pbc) {
            dx = min_image(dx, bx, ibx);
            dy = min_image(dy, by, iby);
            dz = min_image(dz, bz, ibz);
          }
          const Real qq = (dx * dx + dy * dy + dz * dz) * k2;
          const Real q2 = qq * qq;
          const Real sw = rcp_fast<Real>((Real)1 + q2 * qq);
          part += sw;
          const Real gf = c6 * q2 * (sw * sw);
          gx[q] += gf * dx;
          gy[q] += gf * dy;
          gz[q] += gf * dz;
          gjx -= gf * dx;
          gjy -= gf * dy;
          gjz -= gf * dz;
        }
      }
      Real tsum, terr;
      two_sum<Real>(sacc, part, tsum, terr);
      sacc = tsum;
      scomp += terr;
    }
    gjx += __shfl_xor_sync(0xffffffffu, gjx, 1);
    gjy += __shfl_xor_sync(0xffffffffu, gjy, 1);
    gjz += __shfl_xor_sync(0xffffffffu, gjz, 1);
    gjx += __shfl_xor_sync(0xffffffffu, gjx, 2);
    gjy += __shfl_xor_sync(0xffffffffu, gjy, 2);
    gjz += __shfl_xor_sync(0xffffffffu, gjz, 2);
    if (ag == 0 && okj) jB[j] = make_rec<Real>(gjx, gjy, gjz, (Real)0);
  }
  // A gradients: over the warp's B-groups (lanes of one A-group), then warps
  Real *mylig = lig + g.warp * c.na * 3;
#pragma unroll
  for (int q = 0; q < MAXA; ++q) {
    if (4 * q < c.na) {
      Real v[3] = {gx[q], gy[q], gz[q]};
#pragma unroll
      for (int e = 0; e < 3; ++e)
        for (int o = 4; o < 32; o <<= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
      const int i = ag + 4 * q;
      if (g.lane < 4 && i < c.na)
        for (int e = 0; e < 3; ++e) mylig[i * 3 + e] = v[e];
    }
  }
  Real sh, sl;
  two_sum<Real>(sacc, scomp, sh, sl);
  grp_sum_ff<Real>(g, sh, sl, fx->red);
  if (g.t == 0) {
    fx->sh[k] = sh;
    fx->sl[k] = sl;
  }
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

template <typename Real>
__device__ void cv_coord(const Grp &g, GroupFixed<Real> *fx, int k, const typename Rec4<Real>::T *xs,
                         typename Rec4<Real>::T *jA, typename Rec4<Real>::T *jB, Real *lig) {
  if (fx->wd.cv[k].na <= 4 * 10) {
    cv_coord_tiled<Real, 10>(g, fx, k, xs, jA, jB, lig);
    return;
  }
  using R4 = typename Rec4<Real>::T;
  const CvDev &c = fx->wd.cv[k];
  const int32_t *ia = fx->ia[k], *ib = fx->ib[k];
  const Real k2 = (Real)c.inv_r0sq;
  const Real c6 = (Real)-6 * k2;
  const bool pbc = c.pbc != 0;
  const Real bx = (Real)c.box[0], by = (Real)c.box[1], bz = (Real)c.box[2];
  const Real ibx = (Real)c.inv_box[0], iby = (Real)c.inv_box[1], ibz = (Real)c.inv_box[2];
  Real *mylig = lig + g.warp * c.na * 3;
  for (int q = g.lane; q < c.na * 3; q += 32) mylig[q] = 0;
  __syncwarp();
  // this thread's partial sums, compensated (two-sum per term): a CN of
  // thousands must be exact to ~1e-8 relative to place a hill two grid
  // spacings wide, below FP32's resolution. One accumulator per owned B
  // entry keeps the two-sum chains independent.
  constexpr int JB = 4;
  Real sacc[JB], scomp[JB];
#pragma unroll
  for (int jj = 0; jj < JB; ++jj) sacc[jj] = scomp[jj] = 0;
  for (int jb0 = 0; jb0 < c.nb; jb0 += g.G * JB) {
    Real xj[JB], yj[JB], zj[JB], gxj[JB], gyj[JB], gzj[JB], mj[JB];
#pragma unroll
    for (int jj = 0; jj < JB; ++jj) {
      int j = jb0 + jj * g.G + g.t;
      bool ok = j < c.nb;
      R4 p = xs[ib[ok ? j : 0]];
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
        R4 a = xs[ia[oki ? i : 0]];
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
          Real term = m * sw, tsum, terr;
          two_sum<Real>(sacc[jj], term, tsum, terr);
          sacc[jj] = tsum;
          scomp[jj] += terr;
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
  // the per-thread partial sums are combined in hi + lo arithmetic: a CN of
  // a few hundred needs more than FP32's 24 bits to place a hill two grid
  // spacings wide
  Real sh, sl;
  two_sum<Real>(sacc[0], scomp[0], sh, sl);
#pragma unroll
  for (int jj = 1; jj < JB; ++jj) ff_add<Real>(sh, sl, sacc[jj], scomp[jj]);
  grp_sum_ff<Real>(g, sh, sl, fx->red);
  if (g.t == 0) {
    fx->sh[k] = sh;
    fx->sl[k] = sl;
  }
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

// ---------------------------------------------------------------- grid axes

// u = (s - lo) / D = s invD + u0 as hi + lo (FP32 grids: hi + lo floats,
// exact to ~2^-44 relative; FP64 grids: one double).
template <typename Real>
__device__ __forceinline__ void axis_u(const GridDev &gd, int k, Real sh, Real sl, Real &uh, Real &ul);
template <>
__device__ __forceinline__ void axis_u<float>(const GridDev &gd, int k, float sh, float sl, float &uh, float &ul) {
  const float ih = gd.invD_h[k], il = gd.invD_l[k];
  float p = sh * ih;
  float pe = fmaf(sh, ih, -p);  // exact error of the product
  pe = fmaf(sh, il, fmaf(sl, ih, pe));
  float t, te;
  two_sum<float>(p, gd.u0_h[k], t, te);
  te = te + (pe + gd.u0_l[k]);
  uh = t + te;
  ul = te - (uh - t);
}
template <>
__device__ __forceinline__ void axis_u<double>(const GridDev &gd, int k, double sh, double sl, double &uh,
                                               double &ul) {
  uh = fma(sh + sl, gd.invD[k], gd.u0[k]);
  ul = 0;
}

// Split u = uh + ul into a node index a and a fraction f in [0, 1).
template <typename Real>
__device__ __forceinline__ void split_u(Real uh, Real ul, int &a, Real &f) {
  Real fa = floor(uh);
  a = (int)fa;
  f = (uh - fa) + ul;  // uh - fa is exact
  if (f < 0) {
    a -= 1;
    f += 1;
  } else if (f >= 1) {
    a += 1;
    f -= 1;
  }
}

// Per-step axis state of axis k at s = sh + sl: interpolation corners i0/i1
// and weight f (a non-periodic axis clamps s into its range and reports it in
// `clamped`, which zeroes that gradient), and on deposit steps the stencil
// centre i_c = floor(u + 1/2) = da + dc with the fraction df = u - da. Every
// s, finite or not, maps to in-range indices (a non-periodic centre far
// outside is limited to where its box holds no node).
template <typename Real>
struct AxisSt {
  int i0, i1;
  Real f;
  int da, dc, ic_log;
  Real df;
  int clamped;
};

template <typename Real>
__device__ __forceinline__ AxisSt<Real> axis_eval(const GridDev &gd, int R, int k, Real sh, Real sl, bool dep) {
  AxisSt<Real> r;
  r.da = r.dc = r.ic_log = 0;
  r.df = 0;
  r.clamped = 0;
  const int n = gd.n[k];
  const Real rn = (Real)n;
  Real uh, ul;
  axis_u<Real>(gd, k, sh, sl, uh, ul);
  if (gd.periodic[k]) {
    if (!(uh >= 0 && uh < rn)) {
      Real q = floor(uh / rn);
      if (!(q == q) || q > (Real)1e6 || q < (Real)-1e6) {
        uh = 0;
        ul = 0;
      } else {
        ff_add<Real>(uh, ul, -q * rn, (Real)0);
      }
    }
    int a;
    Real f;
    split_u<Real>(uh, ul, a, f);
    if (a >= n) a -= n;
    if (a < 0) a += n;
    if (a < 0 || a >= n) a = 0;
    r.i0 = a;
    r.i1 = (a + 1 == n) ? 0 : a + 1;
    r.f = f;
    if (dep) {
      int c = f >= (Real)0.5 ? 1 : 0;
      r.da = a;
      r.df = f;
      r.dc = c;
      r.ic_log = (a + c == n) ? 0 : a + c;
    }
  } else {
    if (dep) {
      Real dh = uh, dl = ul;
      bool out = false;
      if (!(dh >= (Real)(-R - 2))) {
        dh = (Real)(-R - 2);
        dl = 0;
        out = true;
      }
      if (!(dh <= (Real)(n + R + 1))) {
        dh = (Real)(n + R + 1);
        dl = 0;
        out = true;
      }
      int a;
      Real f;
      split_u<Real>(dh, dl, a, f);
      int c = f >= (Real)0.5 ? 1 : 0;
      r.da = a;
      r.df = f;
      r.dc = c;
      if (out) {
        Real raw = uh + (Real)0.5;
        raw = raw > (Real)1e9 ? (Real)1e9 : (raw < (Real)-1e9 ? (Real)-1e9 : raw);
        r.ic_log = (int)floor(raw == raw ? raw : (Real)0);
      } else {
        r.ic_log = a + c;
      }
    }
    int a;
    Real f;
    if (!(uh >= 0)) {
      a = 0;
      f = 0;
      r.clamped = 1;
    } else if (uh > rn - 1 || (uh == rn - 1 && ul > 0)) {
      a = n - 2;
      f = 1;
      r.clamped = 1;
    } else {
      split_u<Real>(uh, ul, a, f);
      if (a > n - 2) {
        a = n - 2;
        f += 1;
      }
    }
    r.i0 = a;
    r.i1 = a + 1;
    r.f = f;
  }
  return r;
}

// One axis's constants of the interpolation state, held in registers by the
// lane that forms that axis's state every step (the closed-loop form).
template <typename Real>
struct AxisC {
  Real ih, il, u0h, u0l;  // invD and u0 as hi + lo (FP32 grids)
  int n, periodic;
};

template <typename Real>
__device__ __forceinline__ AxisC<Real> axis_consts(const GridDev &gd, int k) {
  AxisC<Real> c;
  if constexpr (sizeof(Real) == 4) {
    c.ih = gd.invD_h[k];
    c.il = gd.invD_l[k];
    c.u0h = gd.u0_h[k];
    c.u0l = gd.u0_l[k];
  } else {
    c.ih = gd.invD[k];
    c.il = 0;
    c.u0h = gd.u0[k];
    c.u0l = 0;
  }
  c.n = gd.n[k];
  c.periodic = gd.periodic[k];
  return c;
}

// The interpolation part of axis_eval (i0, i1, f, clamped) for a step that
// deposits nothing, from register constants and with selects in place of
// the branches of split_u and of the index wrap: the same operations on the
// same values, so the same bits. FP32 grids.
__device__ __forceinline__ AxisSt<float> axis_interp_ff(const AxisC<float> &c, float sh, float sl) {
  AxisSt<float> r;
  r.da = r.dc = r.ic_log = 0;
  r.df = 0;
  float p = sh * c.ih;
  float pe = fmaf(sh, c.ih, -p);
  pe = fmaf(sh, c.il, fmaf(sl, c.ih, pe));
  float t, te;
  two_sum<float>(p, c.u0h, t, te);
  te = te + (pe + c.u0l);
  float uh = t + te, ul = te - (uh - t);
  const float rn = (float)c.n;
  if (c.periodic && !(uh >= 0 && uh < rn)) {
    const float q = floorf(uh / rn);
    if (!(q == q) || q > 1e6f || q < -1e6f) {
      uh = 0;
      ul = 0;
    } else {
      ff_add<float>(uh, ul, -q * rn, 0.f);
    }
  }
  const float fa = floorf(uh);
  int a = (int)fa;
  float f = (uh - fa) + ul;
  const bool neg = f < 0, ge1 = f >= 1;
  a = neg ? a - 1 : (ge1 ? a + 1 : a);
  f = neg ? f + 1 : (ge1 ? f - 1 : f);
  if (c.periodic) {
    a = a >= c.n ? a - c.n : a;
    a = a < 0 ? a + c.n : a;
    a = (a < 0 || a >= c.n) ? 0 : a;
    r.i0 = a;
    r.i1 = a + 1 == c.n ? 0 : a + 1;
    r.f = f;
    r.clamped = 0;
  } else {
    const bool below = !(uh >= 0);
    const bool above = !below && (uh > rn - 1 || (uh == rn - 1 && ul > 0));
    const bool top = a > c.n - 2;
    r.i0 = below ? 0 : ((above || top) ? c.n - 2 : a);
    r.i1 = r.i0 + 1;
    r.f = below ? 0.f : (above ? 1.f : (top ? f + 1 : f));
    r.clamped = (below || above) ? 1 : 0;
  }
  return r;
}

// mABP: the nearest node to s on axis k (from the deposit-step split of u),
// the centre of both the hill and the look-up; wrapped on a periodic axis,
// limited to the grid on a non-periodic one (a limited axis reports
// `clamped` and gets a zero gradient). The hill is centred on the node, so
// its offset within the node is 0.
template <typename Real>
__device__ __forceinline__ void mabp_node(const GridDev &gd, int k, AxisSt<Real> &r) {
  const int n = gd.n[k];
  int c = r.da + r.dc, lim = 0;
  if (gd.periodic[k]) {
    c %= n;
    if (c < 0) c += n;
  } else if (c < 0) {
    c = 0;
    lim = 1;
  } else if (c > n - 1) {
    c = n - 1;
    lim = 1;
  }
  r.da = c;
  r.dc = 0;
  r.df = 0;
  r.ic_log = c;
  r.i0 = r.i1 = c;
  r.f = 0;
  r.clamped = lim;
}

// Axis state for the walker's method (mABP needs the nearest node every step).
template <typename Real>
__device__ __forceinline__ AxisSt<Real> axis_state(const WalkerDev &wd, int k, Real sh, Real sl, bool dep) {
  const bool mabp = wd.method == ABP_METHOD_MABP;
  AxisSt<Real> r = axis_eval<Real>(wd.g, wd.R[k], k, sh, sl, dep || mabp);
  if (mabp) mabp_node<Real>(wd.g, k, r);
  return r;
}

// The group's axis state, one thread per axis (k = g.t < d).
template <typename Real>
__device__ __forceinline__ void axis_setup(GroupFixed<Real> *fx, int k, bool dep) {
  AxisSt<Real> r = axis_state<Real>(fx->wd, k, fx->sh[k], fx->sl[k], dep);
  fx->i0[k] = r.i0;
  fx->i1[k] = r.i1;
  fx->f[k] = r.f;
  if (dep || fx->wd.method == ABP_METHOD_MABP) {
    fx->da[k] = r.da;
    fx->df[k] = r.df;
    fx->dc[k] = r.dc;
    fx->ic_log[k] = r.ic_log;
  }
  if (r.clamped) atomicOr(&fx->clamped, 1 << k);
}

// ---------------------------------------------------------------- the grid tile
//
// A box of T[0] x T[1] x T[2] nodes of the walker's grid, origin org[k],
// held in shared memory with the grid's record layout. The walker's group is
// the grid's only writer, so deposits update the tile and the grid together
// and the tile stays an exact copy; nodes outside the box are read from and
// written to the grid directly.

// Tile-local index of node j along axis k, or -1 outside the box.
__device__ __forceinline__ int tile_rel(const GridDev &gd, const GroupLayout &L, const int *org, int k, int j) {
  int r = j - org[k];
  if (gd.periodic[k]) {
    if (r < 0) r += gd.n[k];
    if (r >= gd.n[k]) r -= gd.n[k];
  }
  return (r >= 0 && r < L.T[k]) ? r : -1;
}

// Thread k: does the box cover what this step needs along axis k (the
// interpolation cell, and the deposit box on deposit steps)? If not, move the
// origin to centre the need and request a reload.
template <typename Real>
__device__ __forceinline__ void tile_check_axis(GroupFixed<Real> *fx, const GroupLayout &L, int k, bool dep) {
  const GridDev &gd = fx->wd.g;
  const int n = gd.n[k], T = L.T[k];
  if (T >= n) return;  // the whole axis is resident (every node has a unique tile index)
  int lo, hi;  // needed node range (unwrapped)
  if (dep) {
    const int R = fx->wd.R[k];
    lo = fx->da[k] + fx->dc[k] - R;
    hi = fx->da[k] + fx->dc[k] + R;
    if (!gd.periodic[k]) {
      lo = max(lo, 0);
      hi = min(hi, n - 1);
      if (lo > hi) lo = hi = fx->i0[k];  // box entirely outside: nothing to hold
      lo = min(lo, fx->i0[k]);
      hi = max(hi, fx->i0[k] + 1);
    }
  } else {
    lo = fx->i0[k];
    hi = fx->i0[k] + 1;
  }
  int span = hi - lo + 1;
  int r = lo - fx->org[k];
  if (gd.periodic[k]) {
    r %= n;
    if (r < 0) r += n;
  }
  if (r >= 0 && r + span <= T) return;
  int o = lo - (T - span) / 2;
  if (gd.periodic[k]) {
    o %= n;
    if (o < 0) o += n;
  } else {
    o = max(0, min(o, n - T));
  }
  fx->org[k] = o;
  fx->reload = 1;
}

// All group threads: copy the box from the grid (cp.async, 16 B pieces),
// one axis-0 row at a time (a row is contiguous in the grid unless it wraps
// around a periodic axis 0, where it splits in two).
template <typename Real>
__device__ void tile_load(const Grp &g, GroupFixed<Real> *fx, const GroupLayout &L, unsigned char *tile) {
  const GridDev &gd = fx->wd.g;
  const int rb = gd.rec_bytes;
  const int T0 = L.T[0], T1 = gd.d > 1 ? L.T[1] : 1, T2 = gd.d > 2 ? L.T[2] : 1;
  const int n0 = gd.n[0];
  const int o0 = fx->org[0];
  const int first = min(T0, n0 - o0);  // nodes before the wrap of axis 0
  const int pieces_row = T0 * rb / 16, first_pieces = first * rb / 16;
  const unsigned char *grid = reinterpret_cast<const unsigned char *>(gd.rec);
  int j1 = fx->org[1], j2 = fx->org[2];
  for (int r2 = 0; r2 < T2; ++r2) {
    int jj1 = j1;
    for (int r1 = 0; r1 < T1; ++r1) {
      const unsigned char *row =
          grid + chk_node(gd, (long long)j2 * (gd.d > 1 ? gd.n[1] : 1) * n0 + (long long)jj1 * n0) * rb;
      unsigned char *dst = tile + ((size_t)r2 * T1 + r1) * T0 * rb;
      for (int p = g.t; p < pieces_row; p += g.G) {
        const unsigned char *src =
            p < first_pieces ? row + (size_t)o0 * rb + p * 16 : row + (size_t)(p - first_pieces) * 16;
        cp_async16(dst + p * 16, src);
      }
      if (++jj1 == gd.n[1]) jj1 = 0;
    }
    if (++j2 == gd.n[2]) j2 = 0;
  }
  cp_async_commit();
  cp_async_wait_all();
  g.sync();
}

// ---------------------------------------------------------------- node access

// 1 + d values (value + compensation) of a node record at p.
template <typename Acc>
__device__ __forceinline__ void rec_values(const GridDev &gd, const unsigned char *p, Acc *v) {
  if (gd.prec == ABP_PREC_FP32_COMP) {
    if (gd.d == 1) {
      float4 r = *reinterpret_cast<const float4 *>(p);
      v[0] = (Acc)r.x + (Acc)r.z;
      v[1] = (Acc)r.y + (Acc)r.w;
    } else {
      const float4 *q = reinterpret_cast<const float4 *>(p);
      float4 a = q[0], b = q[1];
      v[0] = (Acc)a.x + (Acc)b.x;
      v[1] = (Acc)a.y + (Acc)b.y;
      v[2] = (Acc)a.z + (Acc)b.z;
      v[3] = (Acc)a.w + (Acc)b.w;
    }
  } else {
    if (gd.d == 1) {
      double2 r = *reinterpret_cast<const double2 *>(p);
      v[0] = (Acc)r.x;
      v[1] = (Acc)r.y;
    } else {
      D4 r = *reinterpret_cast<const D4 *>(p);
      v[0] = (Acc)r.x;
      v[1] = (Acc)r.y;
      v[2] = (Acc)r.z;
      v[3] = (Acc)r.w;
    }
  }
}

// Address of corner `lane` (bit k selects i1 on axis k) in the tile or grid.
template <typename Real, bool TILE>
__device__ __forceinline__ const unsigned char *corner_ptr(const GroupFixed<Real> *fx, const GroupLayout &L,
                                                           const unsigned char *tile, int lane) {
  const GridDev &gd = fx->wd.g;
  long long node = 0, mul = 1;
  for (int k = 0; k < gd.d; ++k) {
    int j = ((lane >> k) & 1) ? fx->i1[k] : fx->i0[k];
    if (TILE) {
      int r = tile_rel(gd, L, fx->org, k, j);
      node += mul * r;
      mul *= L.T[k];
    } else {
      node += mul * j;
      mul *= gd.n[k];
    }
  }
  return TILE ? tile + node * gd.rec_bytes
              : reinterpret_cast<const unsigned char *>(gd.rec) + chk_node(gd, node) * gd.rec_bytes;
}

// a2: V_b(s_t) from the grid before the deposit, in FP64, by warp 0's first
// 2^d lanes; returns the value in lane 0.
template <typename Real, bool TILE>
__device__ __forceinline__ double height_interp(const GroupFixed<Real> *fx, const GroupLayout &L,
                                                const unsigned char *tile, int lane) {
  const GridDev &gd = fx->wd.g;
  double acc = 0;
  if (lane < (1 << gd.d)) {
    double w = 1;
    for (int k = 0; k < gd.d; ++k) {
      double f = (double)fx->f[k];
      w *= ((lane >> k) & 1) ? f : 1.0 - f;
    }
    double v[4];
    rec_values<double>(gd, corner_ptr<Real, TILE>(fx, L, tile, lane), v);
    acc = w * v[0];
  }
  for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// mABP's compact hill (Eq. (compacthill)) at the node-to-centre distance
// `dist` along one CV, S = e^p e^(-p / (1 - x^2)) = e^(-p x^2 / (1 - x^2)),
// x = dist / a (0 for |x| >= 1), and the factor that turns the deposit's S
// into its derivative along the grid coordinate:
// d S(xi* - xi) / d xi = S (-2 p dist / (a^2 (1 - x^2)^2)).
template <typename Real>
__device__ __forceinline__ void compact_factors(Real dist, Real a, int p, Real &S, Real &Dfac) {
  const Real x = dist / a;
  if (!(fabs(x) < (Real)1)) {
    S = 0;
    Dfac = 0;
    return;
  }
  const Real om = (Real)1 - x * x;
  S = exp(-(Real)p * x * x / om);
  Dfac = (Real)-2 * (Real)p * dist / (a * a * om * om);
}

// a3 (part 1): per-axis factor tables of the stencil box around s: node index
// j = i_c - R + o (or -1 outside a non-periodic axis), G_k = exp(-d^2 / 2 sigma^2)
// and -d / sigma^2, d = (j - u) D the node-to-centre distance, formed as
// ((dc - R + o) - df) D from the small exact parts of u.
template <typename Real>
__device__ void build_tables(const Grp &g, GroupFixed<Real> *fx) {
  const WalkerDev &wd = fx->wd;
  const GridDev &gd = wd.g;
  const bool mabp = wd.method == ABP_METHOD_MABP;
  for (int k = 0; k < gd.d; ++k) {
    const int R = wd.R[k], span = 2 * R + 1, n = gd.n[k];
    const int a = fx->da[k], c = fx->dc[k];
    const Real f = fx->df[k], D = (Real)gd.D[k];
    const Real i2 = (Real)wd.inv2s2[k], is2 = (Real)wd.invs2[k];
    const Real ak = (Real)wd.a[k];
    for (int o = g.t; o < span; o += g.G) {
      int rel = c - R + o;
      int j = a + rel;
      Real dist = ((Real)rel - f) * D;
      int jj = j;
      if (gd.periodic[k]) {
        jj = j % n;
        if (jj < 0) jj += n;
      } else if (j < 0 || j >= n) {
        jj = -1;
      }
      fx->tabJ[k][o] = jj;
      if (mabp) {
        compact_factors<Real>(dist, ak, wd.p, fx->tabG[k][o], fx->tabD[k][o]);
      } else {
        fx->tabG[k][o] = exp(-dist * dist * i2);
        fx->tabD[k][o] = -dist * is2;
      }
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

// Apply h G (and its derivative terms) to one node record held in two
// 16-byte halves a, b (b unused for 16-byte records).
template <typename Real>
__device__ __forceinline__ void rmw_regs(int d, float4 &a, float4 &b, Real G, Real d0, Real d1, Real d2);
template <>
__device__ __forceinline__ void rmw_regs<float>(int d, float4 &a, float4 &b, float G, float d0, float d1, float d2) {
  if (d == 1) {
    two_sum_add(a.x, a.z, G);
    two_sum_add(a.y, a.w, __fmul_rn(G, d0));
  } else {
    two_sum_add(a.x, b.x, G);
    two_sum_add(a.y, b.y, __fmul_rn(G, d0));
    two_sum_add(a.z, b.z, __fmul_rn(G, d1));
    if (d > 2) two_sum_add(a.w, b.w, __fmul_rn(G, d2));
  }
}
template <>
__device__ __forceinline__ void rmw_regs<double>(int d, float4 &a, float4 &b, double G, double d0, double d1,
                                                 double d2) {
  union U {
    float4 f;
    double2 v;
  };
  U ua, ub;
  ua.f = a;
  ub.f = b;
  ua.v.x += G;
  ua.v.y += G * d0;
  if (d > 1) ub.v.x += G * d1;
  if (d > 2) ub.v.y += G * d2;
  a = ua.f;
  b = ub.f;
}

template <typename Real>
__device__ __forceinline__ void rmw_node(const GridDev &gd, unsigned char *p, Real G, Real d0, Real d1, Real d2) {
  float4 *q = reinterpret_cast<float4 *>(p);
  float4 a = q[0], b = gd.rec_bytes == 32 ? q[1] : make_float4(0, 0, 0, 0);
  rmw_regs<Real>(gd.d, a, b, G, d0, d1, d2);
  q[0] = a;
  if (gd.rec_bytes == 32) q[1] = b;
}

// a3 (part 2): add h G and h G (-d_k / sigma_k^2) at every in-range node of
// the box. FP32_COMP grids accumulate with two-sum compensation; FP64 grids
// add directly. With a tile, nodes inside it are updated in shared memory and
// the result stored to the grid; other nodes are updated in the grid.
template <typename Real, bool TILE, int UNR = 4>
__device__ void deposit_stencil(const Grp &g, GroupFixed<Real> *fx, const GroupLayout &L, unsigned char *tile) {
  const WalkerDev &wd = fx->wd;
  const GridDev &gd = wd.g;
  const int d = gd.d, rb = gd.rec_bytes;
  const int s0 = 2 * wd.R[0] + 1;
  const int s1 = d > 1 ? 2 * wd.R[1] + 1 : 1;
  const int s2 = d > 2 ? 2 * wd.R[2] + 1 : 1;
  const int total = s0 * s1 * s2;
  const Real h = fx->hf;
  const long long n0 = gd.n[0], n01 = (long long)gd.n[0] * (d > 1 ? gd.n[1] : 1);
  unsigned char *grid = reinterpret_cast<unsigned char *>(gd.rec);
  // thread t visits box nodes t, t + G, ... (axis 0 fastest); the box index
  // (o0, o1, o2) advances incrementally instead of by division
  int o0 = g.t, o1 = 0, o2 = 0;
  while (o0 >= s0) {
    o0 -= s0;
    if (++o1 == s1) {
      o1 = 0;
      ++o2;
    }
  }
  const int step0 = g.G % s0, step1 = g.G / s0;
  auto advance = [&]() {
    o0 += step0;
    o1 += step1;
    if (o0 >= s0) {
      o0 -= s0;
      ++o1;
    }
    while (o1 >= s1) {
      o1 -= s1;
      ++o2;
    }
  };
  // UNR nodes per round: their records are loaded before any is updated, so
  // the grid reads of a round overlap
  for (int base = g.t; base < total; base += UNR * g.G) {
    unsigned char *ptr[UNR];
    bool intile[UNR];
    Real Gv[UNR], d0v[UNR], d1v[UNR], d2v[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      ptr[u] = nullptr;
      intile[u] = false;
      Gv[u] = d0v[u] = d1v[u] = d2v[u] = 0;
      if (u > 0) advance();
      if (base + u * g.G >= total) continue;
      int j0 = fx->tabJ[0][o0];
      int j1 = d > 1 ? fx->tabJ[1][o1] : 0;
      int j2 = d > 2 ? fx->tabJ[2][o2] : 0;
      if ((j0 | j1 | j2) < 0) continue;
      Real G = h * fx->tabG[0][o0];
      if (d > 1) G = G * fx->tabG[1][o1];
      if (d > 2) G = G * fx->tabG[2][o2];
      Gv[u] = G;
      d0v[u] = fx->tabD[0][o0];
      d1v[u] = d > 1 ? fx->tabD[1][o1] : (Real)0;
      d2v[u] = d > 2 ? fx->tabD[2][o2] : (Real)0;
      ptr[u] = grid + chk_node(gd, (long long)j0 + (long long)n0 * j1 + (long long)n01 * j2) * rb;
      if (TILE) {
        int t0 = tile_rel(gd, L, fx->org, 0, j0);
        int t1 = d > 1 ? tile_rel(gd, L, fx->org, 1, j1) : 0;
        int t2 = d > 2 ? tile_rel(gd, L, fx->org, 2, j2) : 0;
        if ((t0 | t1 | t2) >= 0) {
          unsigned char *tp = tile + (t0 + L.T[0] * (t1 + (d > 1 ? L.T[1] : 1) * t2)) * rb;
          rmw_node<Real>(gd, tp, G, d0v[u], d1v[u], d2v[u]);
          const float4 *src = reinterpret_cast<const float4 *>(tp);
          float4 *dst = reinterpret_cast<float4 *>(ptr[u]);
          dst[0] = src[0];
          if (rb == 32) dst[1] = src[1];
          intile[u] = true;
        }
      }
    }
    advance();  // to this thread's first node of the next round
    // grid nodes outside the tile: load all, then update all
    float4 ra[UNR], rbv[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (ptr[u] && !intile[u]) {
        const float4 *q = reinterpret_cast<const float4 *>(ptr[u]);
        ra[u] = q[0];
        rbv[u] = rb == 32 ? q[1] : make_float4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      if (!ptr[u] || intile[u]) continue;
      rmw_regs<Real>(d, ra[u], rbv[u], Gv[u], d0v[u], d1v[u], d2v[u]);
      float4 *q = reinterpret_cast<float4 *>(ptr[u]);
      q[0] = ra[u];
      if (rb == 32) q[1] = rbv[u];
    }
  }
}

// ---------------------------------------------------------------- a4 + a5

// mABP: the bias and its gradient from the histograms at the nearest node,
// V = kT b/(1-b) ln(c (1-b) h + 1) (Eq. (apfm)) and
// dV/dxi_k = c b kT h'_k / (1 + c (1-b) h) (Eq. (btraj-grad)).
template <typename Real>
__device__ __forceinline__ void mabp_bias(const WalkerDev &wd, const Real *acc, Real &V, Real *dv) {
  const Real hh = acc[0], ch = (Real)wd.mabp_h * hh;
  V = (Real)wd.mabp_k * log1p(ch);
  const Real den = (Real)1 + ch;
  for (int k = 0; k < wd.g.d; ++k) dv[k] = (Real)wd.mabp_g * acc[1 + k] / den;
}

// dU/ds_k of the CV range limit: kwall (s - smax_k) above smax_k, else 0.
template <typename Real>
__device__ __forceinline__ Real wall_grad(const WalkerDev &wd, int k, Real s) {
  if constexpr (sizeof(Real) == 4)
    return (wd.kwall_f > 0.f && s > wd.smax_f[k]) ? wd.kwall_f * (s - wd.smax_f[k]) : 0.f;
  else
    return (wd.kwall > 0 && s > (Real)wd.smax[k]) ? (Real)wd.kwall * (s - (Real)wd.smax[k]) : (Real)0;
}

// a4: V and dV/ds_k at s after the deposit, by warp 0's first 2^d lanes,
// combined with a fixed xor-butterfly; a clamped axis gets a zero gradient.
// (For mABP the corners all sit on the nearest node with weight 1 on the
// first, which yields that node's histograms, turned into the bias.)
template <typename Real, bool TILE>
__device__ void interp_step(const Grp &g, GroupFixed<Real> *fx, const GroupLayout &L, const unsigned char *tile) {
  const GridDev &gd = fx->wd.g;
  if (g.warp == 0) {
    Real acc[4] = {0, 0, 0, 0};
    if (g.lane < (1 << gd.d)) {
      Real w = 1;
      for (int k = 0; k < gd.d; ++k) w *= ((g.lane >> k) & 1) ? fx->f[k] : (Real)1 - fx->f[k];
      Real v[4];
      rec_values<Real>(gd, corner_ptr<Real, TILE>(fx, L, tile, g.lane), v);
      for (int q = 0; q <= gd.d; ++q) acc[q] = w * v[q];
    }
    for (int q = 0; q < 4; ++q)
      for (int o = 1; o < 8; o <<= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (g.lane == 0) {
      if (fx->wd.method == ABP_METHOD_MABP) {
        Real V, dvm[3];
        mabp_bias<Real>(fx->wd, acc, V, dvm);
        acc[0] = V;
        for (int k = 0; k < gd.d; ++k) acc[1 + k] = dvm[k];
      }
      fx->V = acc[0];
      for (int k = 0; k < gd.d; ++k) {
        Real dv = ((fx->clamped >> k) & 1) ? (Real)0 : acc[1 + k];
        dv += wall_grad<Real>(fx->wd, k, fx->sh[k] + fx->sl[k]);
        fx->dvds[k] = dv;
        fx->dV[k] = dv;
      }
      if (fx->clamped) fx->flags |= ABP_WFLAG_OOR;
    }
  }
  g.sync();
}

// a5: F_i = - sum_k dV/ds_k ds_k/dx_i into the force accumulators fs (zeroed
// by the caller). Lists are unique, and each list is a separate phase, so
// every accumulator is updated in a fixed order.
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
    const int32_t *ia = fx->ia[k], *ib = fx->ib[k];
    Real dv = fx->dvds[k];
    if (c.type == ABP_CV_COM_DIST) {
      const Real *wa = fx->wa[k], *wb = fx->wb[k];
      Real ux = fx->com_u[k][0] * dv, uy = fx->com_u[k][1] * dv, uz = fx->com_u[k][2] * dv;
      for (int i = g.t; i < c.na; i += g.G) {
        Real w = wa[i];
        R4 &f = fs[ia[i]];
        f.x += w * ux;
        f.y += w * uy;
        f.z += w * uz;
      }
      g.sync();
      for (int i = g.t; i < c.nb; i += g.G) {
        Real w = wb[i];
        R4 &f = fs[ib[i]];
        f.x -= w * ux;
        f.y -= w * uy;
        f.z -= w * uz;
      }
      g.sync();
    } else if (c.type == ABP_CV_DIHEDRAL) {
      if (g.t < 4) {
        R4 &f = fs[ia[g.t]];
        f.x -= dv * fx->dih_g[k][g.t][0];
        f.y -= dv * fx->dih_g[k][g.t][1];
        f.z -= dv * fx->dih_g[k][g.t][2];
      }
      g.sync();
    } else {
      const R4 *jA = reinterpret_cast<const R4 *>(cur);
      const R4 *jB = jA + c.na;
      for (int i = g.t; i < c.na; i += g.G) {
        R4 &f = fs[ia[i]];
        R4 j = jA[i];
        f.x -= dv * j.x;
        f.y -= dv * j.y;
        f.z -= dv * j.z;
      }
      g.sync();
      for (int i = g.t; i < c.nb; i += g.G) {
        R4 &f = fs[ib[i]];
        R4 j = jB[i];
        f.x -= dv * j.x;
        f.y -= dv * j.y;
        f.z -= dv * j.z;
      }
      g.sync();
      cur += (c.na + c.nb) * rsz + align32(g.nwarps * c.na * 3 * (int)sizeof(Real));
    }
  }
}

}  // namespace abp
