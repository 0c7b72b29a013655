// abp_window_ops.cuh -- per-step operations of the windowed form, one thread
// (or one lane pair) per task: a step's CVs and Jacobian factors, its axis
// state, the corner reads and the multilinear combination of a4, the height
// of a2 from the corner records, and a5 from an atom's term list. The
// windowed form (abp_kernels.cu) and the closed-loop form (abp_md.cu) both
// run a step through these functions, so the two compute a step's bias
// force and deposits with the same arithmetic.
#pragma once

#include "abp_device.cuh"

namespace abp {

template <typename Real>
__device__ __forceinline__ bool finite_rec(const typename Rec4<Real>::T &p) {
  return isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
}

template <typename Real>
__device__ __forceinline__ void store_force(typename Rec4<Real>::T *fo, const typename Rec4<Real>::T &f, int mode) {
  if (mode == ABP_FORCES_ACCUMULATE) {
    typename Rec4<Real>::T o = *fo;
    o.x += f.x;
    o.y += f.y;
    o.z += f.z;
    *fo = o;
  } else {
    *fo = make_rec<Real>(f.x, f.y, f.z, 0);
  }
}

// (j, i) = divmod(t, n), advanced by G each time without a division.
struct Iter2 {
  int j, i, q, r, n;
  __device__ __forceinline__ Iter2(int t, int G, int n_) : n(n_) {
    j = t / n;
    i = t - j * n;
    q = G / n;
    r = G - q * n;
  }
  __device__ __forceinline__ void next() {
    i += r;
    j += q;
    if (i >= n) {
      i -= n;
      ++j;
    }
  }
};

// Rounded arithmetic with no contraction left to the compiler, so that every
// inlined copy of a CV computes the same bits.
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// One group's part of a COM distance: the group's first atom r0 and the
// weighted offsets of its atoms from r0, summed in list order (FP32 walkers:
// compensated, the low part of the sum in lo; FP64 walkers: lo = 0).
template <typename Real>
__device__ __forceinline__ void com_sum(const int32_t *list, const Real *wts, int n,
                                        const typename Rec4<Real>::T *x, Real *r0, Real *acc, Real *lo) {
  const auto p0 = x[list[0]];
  Real a0 = 0, a1 = 0, a2 = 0, c0 = 0, c1 = 0, c2 = 0;
#pragma unroll 4
  for (int i = 0; i < n; ++i) {
    Real w = wts[i];
    auto p = x[list[i]];
    if constexpr (sizeof(Real) == 4) {
      // Kahan: c holds minus the low part the running sum has lost
      const Real y0 = fma_rn(w, sub_rn(p.x, p0.x), -c0), y1 = fma_rn(w, sub_rn(p.y, p0.y), -c1),
                 y2 = fma_rn(w, sub_rn(p.z, p0.z), -c2);
      const Real t0 = add_rn(a0, y0), t1 = add_rn(a1, y1), t2 = add_rn(a2, y2);
      c0 = sub_rn(sub_rn(t0, a0), y0);
      c1 = sub_rn(sub_rn(t1, a1), y1);
      c2 = sub_rn(sub_rn(t2, a2), y2);
      a0 = t0;
      a1 = t1;
      a2 = t2;
    } else {
      a0 = fma_rn(w, sub_rn(p.x, p0.x), a0);
      a1 = fma_rn(w, sub_rn(p.y, p0.y), a1);
      a2 = fma_rn(w, sub_rn(p.z, p0.z), a2);
    }
  }
  r0[0] = p0.x;
  r0[1] = p0.y;
  r0[2] = p0.z;
  acc[0] = a0;
  acc[1] = a1;
  acc[2] = a2;
  lo[0] = -c0;
  lo[1] = -c1;
  lo[2] = -c2;
}

// The end of a COM distance from the two groups' parts: s = |R_B - R_A|
// (minimum image in a periodic box), as sh + sl for FP32 walkers
// (com_finish_ff), and u = d / s.
template <typename Real>
__device__ __forceinline__ int com_finish(const CvDev &c, const Real *ra, const Real *a, const Real *al,
                                          const Real *rb, const Real *b, const Real *bl, Real &s, Real &sl, Real *u) {
  if constexpr (sizeof(Real) == 4) {
    return com_finish_ff(c, ra, a, al, rb, b, bl, s, sl, u);
  } else {
    Real d[3];
    for (int q = 0; q < 3; ++q) d[q] = add_rn(sub_rn(rb[q], ra[q]), sub_rn(b[q], a[q]));
    if (c.pbc)
      for (int q = 0; q < 3; ++q) d[q] = min_image(d[q], c.box[q], c.inv_box[q]);
    Real r = sqrt(fma_rn(d[2], d[2], fma_rn(d[1], d[1], mul_rn(d[0], d[0]))));
    s = r;
    sl = 0;
    if (r > 0) {
      Real ir = rcp_fast<Real>(r);
      for (int q = 0; q < 3; ++q) u[q] = mul_rn(d[q], ir);
      return 0;
    }
    for (int q = 0; q < 3; ++q) u[q] = 0;
    return ABP_WFLAG_SINGULAR;
  }
}

// COM distance of one step by one thread: each group's weighted offsets from
// its first atom summed in list order, then s = |R_B - R_A| and u = d / s.
template <typename Real>
__device__ __forceinline__ int com_thread(const CvDev &c, const int32_t *ia, const int32_t *ib, const Real *wa,
                                          const Real *wb, const typename Rec4<Real>::T *x, Real &s, Real &sl,
                                          Real *u) {
  Real ra[3], a[3], al[3], rb[3], b[3], bl[3];
  com_sum<Real>(ia, wa, c.na, x, ra, a, al);
  com_sum<Real>(ib, wb, c.nb, x, rb, b, bl);
  return com_finish<Real>(c, ra, a, al, rb, b, bl, s, sl, u);
}

// The end of a4 for one step: V and dV/dxi from the interpolated fields (for
// mABP, the nearest node's histograms turned into the bias), a zero gradient
// on a clamped axis, and the Jacobian factors scaled for a5.
template <typename Real>
__device__ __forceinline__ void finish_lookup(const WalkerDev &wd, StepRec<Real> &st, Real *acc) {
  const int d = wd.g.d;
  if (wd.method == ABP_METHOD_MABP) {
    Real V, dvm[3] = {0, 0, 0};
    mabp_bias<Real>(wd, acc, V, dvm);
    acc[0] = V;
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[1 + k] = dvm[k];
  }
  st.V = acc[0];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < d) {
      const Real dv = (((st.clamped >> k) & 1) ? (Real)0 : acc[1 + k]) + wall_grad<Real>(wd, k, st.s[k]);
      st.dv[k] = dv;
      const int nj = wd.cv[k].type == ABP_CV_COM_DIST ? 3 : 12;
      for (int q = 0; q < nj; ++q) st.jac[k][q] *= dv;
    }
}

// A node record as two 16-byte halves: both for the 32-byte records of a
// 2D or 3D grid, the first for the 16-byte records of a 1D grid.
template <int DIM>
__device__ __forceinline__ void rec_load(const unsigned char *p, float4 &a, float4 &b) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
  a = q[0];
  b = DIM > 1 ? q[1] : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The 1 + d values of a record held in registers, formed as rec_values forms
// them from memory: an FP32 grid (Real = float) holds value + compensation
// per field, an FP64 grid (Real = double) the values.
template <typename Real, int DIM, typename Acc>
__device__ __forceinline__ void rec_vals(const float4 &a, const float4 &b, Acc *v) {
  if constexpr (sizeof(Real) == 4) {
    if constexpr (DIM == 1) {
      v[0] = (Acc)a.x + (Acc)a.z;
      v[1] = (Acc)a.y + (Acc)a.w;
    } else {
      v[0] = (Acc)a.x + (Acc)b.x;
      v[1] = (Acc)a.y + (Acc)b.y;
      v[2] = (Acc)a.z + (Acc)b.z;
      if (DIM > 2) v[3] = (Acc)a.w + (Acc)b.w;
    }
  } else {
    union U {
      float4 f;
      double2 v;
    };
    U ua, ub;
    ua.f = a;
    ub.f = b;
    v[0] = (Acc)ua.v.x;
    v[1] = (Acc)ua.v.y;
    if (DIM > 1) v[2] = (Acc)ub.v.x;
    if (DIM > 2) v[3] = (Acc)ub.v.y;
  }
}

// Grid node of corner c of a step (bit k of c selects i1 on axis k).
template <typename Real, int DIM>
__device__ __forceinline__ long long corner_node(const GridDev &gd, const StepRec<Real> &st, int c) {
  long long node = 0, mul = 1;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    node += mul * (((c >> k) & 1) ? st.i1[k] : st.i0[k]);
    mul *= gd.n[k];
  }
  return node;
}

// Multilinear weight of corner c.
template <typename Real, int DIM>
__device__ __forceinline__ Real corner_weight(const StepRec<Real> &st, int c) {
  Real wc = 1;
#pragma unroll
  for (int k = 0; k < DIM; ++k) wc *= ((c >> k) & 1) ? st.f[k] : (Real)1 - st.f[k];
  return wc;
}

template <int DIM>
__device__ __forceinline__ const unsigned char *node_ptr(const GridDev &gd, long long node) {
  return reinterpret_cast<const unsigned char *>(gd.rec) + chk_node(gd, node) * (DIM > 1 ? 32 : 16);
}

// a4 of one step, part 1: the 2^d corners' records, loaded together.
template <typename Real, int DIM>
__device__ __forceinline__ void interp_load(const WalkerDev &wd, const StepRec<Real> &st, float4 *ca, float4 *cb) {
#pragma unroll
  for (int c = 0; c < (1 << DIM); ++c) rec_load<DIM>(node_ptr<DIM>(wd.g, corner_node<Real, DIM>(wd.g, st, c)), ca[c], cb[c]);
}

// a4 of one step, part 2: the corners combined in corner order.
template <typename Real, int DIM>
__device__ __forceinline__ void interp_combine(const WalkerDev &wd, StepRec<Real> &st, const float4 *ca,
                                               const float4 *cb) {
  Real acc[4] = {0, 0, 0, 0};
#pragma unroll
  for (int c = 0; c < (1 << DIM); ++c) {
    const Real wc = corner_weight<Real, DIM>(st, c);
    Real v[4];
    rec_vals<Real, DIM>(ca[c], cb[c], v);
#pragma unroll
    for (int q = 0; q <= DIM; ++q) acc[q] += wc * v[q];
  }
  finish_lookup<Real>(wd, st, acc);
}

// a4 of one step: the 2^d corners' records loaded together, then combined in
// corner order.
template <typename Real, int DIM>
__device__ __forceinline__ void interp_one(const WalkerDev &wd, StepRec<Real> &st) {
  constexpr int NC = 1 << DIM;
  Real v[NC][4];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    float4 a, b;
    rec_load<DIM>(node_ptr<DIM>(wd.g, corner_node<Real, DIM>(wd.g, st, c)), a, b);
    rec_vals<Real, DIM>(a, b, v[c]);
  }
  Real acc[4] = {0, 0, 0, 0};
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const Real wc = corner_weight<Real, DIM>(st, c);
#pragma unroll
    for (int q = 0; q <= DIM; ++q) acc[q] += wc * v[c][q];
  }
  finish_lookup<Real>(wd, st, acc);
}

// RMSD of one step by one thread (SI "Definition of the RMSD"):
// s = (sum_i |x_i - x0_i|^2 / N + 0.01)^(1/2), no fit, and ds/dx_i =
// (x_i - x0_i) / (N s) for the N <= 4 atoms into J[3 i ..].
template <typename Real>
__device__ __forceinline__ int rmsd_thread(const CvDev &c, const int32_t *ia, const typename Rec4<Real>::T *x,
                                           Real &s, Real *J) {
  const Real *ref;
  if constexpr (sizeof(Real) == 4)
    ref = c.ref;
  else
    ref = c.ref64;
  Real dx[4][3], acc = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < c.na) {
      const auto p = x[ia[i]];
      dx[i][0] = p.x - ref[3 * i];
      dx[i][1] = p.y - ref[3 * i + 1];
      dx[i][2] = p.z - ref[3 * i + 2];
      acc += dx[i][0] * dx[i][0] + dx[i][1] * dx[i][1] + dx[i][2] * dx[i][2];
    }
  const Real N = (Real)c.na;
  s = sqrt(acc / N + (Real)0.01);
  const Real inv = (Real)1 / (N * s);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (i < c.na)
      for (int q = 0; q < 3; ++q) J[3 * i + q] = dx[i][q] * inv;
  return 0;
}

// The step record's CV k: the value, flags and axis state.
template <typename Real>
__device__ __forceinline__ void window_cv_rec(const WalkerDev &wd, int k, Real sk, Real slk, int fl, bool dep,
                                              StepRec<Real> &st) {
  st.s[k] = sk;
  st.sl[k] = slk;
  AxisSt<Real> ax = axis_state<Real>(wd, k, sk, slk, dep);
  st.i0[k] = ax.i0;
  st.i1[k] = ax.i1;
  st.f[k] = ax.f;
  st.da[k] = ax.da;
  st.dc[k] = ax.dc;
  st.df[k] = ax.df;
  st.ic_log[k] = ax.ic_log;
  st.cfl[k] = fl | (ax.clamped << 16);
}

// Phase A task: CV k of one step (row x of the window), its Jacobian
// factors and axis state.
template <typename Real>
__device__ __forceinline__ void window_cv(const GroupFixed<Real> *fx, const typename Rec4<Real>::T *x, int k,
                                          bool dep, StepRec<Real> &st) {
  const WalkerDev &wd = fx->wd;
  const CvDev &c = wd.cv[k];
  Real sk, slk = 0;
  int fl;
  if (c.type == ABP_CV_COM_DIST)
    fl = com_thread<Real>(c, fx->ia[k], fx->ib[k], fx->wa[k], fx->wb[k], x, sk, slk, st.jac[k]);
  else if (c.type == ABP_CV_DIHEDRAL)
    fl = dihedral_eval<Real>(c, fx->ia[k], x, sk, reinterpret_cast<Real(*)[3]>(st.jac[k]), slk);
  else
    fl = rmsd_thread<Real>(c, fx->ia[k], x, sk, st.jac[k]);
  window_cv_rec<Real>(wd, k, sk, slk, fl, dep, st);
}

// A COM-distance task of the windowed form on two lanes (2i: group A, 2i + 1:
// group B, the same sums as com_thread's), finished by the even lane. Every
// lane of the warp calls it (the odd lanes' parts travel by shuffle); `live`
// is false on lanes past the window's steps.
template <typename Real>
__device__ __forceinline__ void window_com2(const GroupFixed<Real> *fx, const typename Rec4<Real>::T *x, int k,
                                            bool dep, bool live, bool odd, StepRec<Real> &st) {
  const WalkerDev &wd = fx->wd;
  const CvDev &c = wd.cv[k];
  Real r0[3], acc[3], lo[3];
  if (odd)
    com_sum<Real>(fx->ib[k], fx->wb[k], c.nb, x, r0, acc, lo);
  else
    com_sum<Real>(fx->ia[k], fx->wa[k], c.na, x, r0, acc, lo);
  Real o0[3], oa[3], ol[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    o0[q] = __shfl_xor_sync(0xffffffffu, r0[q], 1);
    oa[q] = __shfl_xor_sync(0xffffffffu, acc[q], 1);
    ol[q] = __shfl_xor_sync(0xffffffffu, lo[q], 1);
  }
  if (odd || !live) return;
  Real sk, slk;
  const int fl = com_finish<Real>(c, r0, acc, lo, o0, oa, ol, sk, slk, st.jac[k]);
  window_cv_rec<Real>(wd, k, sk, slk, fl, dep, st);
}

// a2's end: V_b(s_t) from the corner terms t (pairwise, in corner order), the
// height, and the deposit log record.
template <typename Real>
__device__ __forceinline__ void window_height_out(GroupFixed<Real> *fx, const StepRec<Real> &st, const double *t,
                                                  long long step, const DepositLog &log) {
  const WalkerDev &wd = fx->wd;
  const int d = wd.g.d, nc = wd.method == ABP_METHOD_MABP ? 0 : 1 << d;
  const double V0 = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
  const double h = nc ? wd.w * exp(-V0 * wd.inv_dT) : wd.w;
  fx->hV = V0;
  fx->hf = (Real)h;
  if (log.rec) {
    unsigned long long slot = atomicAdd(log.count, 1ull);
    if (slot < log.cap) {
      abp_deposit_rec r;
      r.step = step;
      r.walker_id = wd.id;
      for (int k = 0; k < 3; ++k) {
        r.ic[k] = k < d ? st.ic_log[k] : 0;
        r.s[k] = k < d ? (double)st.s[k] + (double)st.sl[k] : 0.0;
      }
      r.height = h;
      log.rec[slot] = r;
    }
  }
}

// a2 of a window deposit, by one thread, from the deposit step's 2^d corner
// records before the deposit: V_b(s_t) in FP64 (the corners' value fields,
// combined pairwise in corner order), the height h = w exp(-V / dT), and the
// deposit log record.
template <typename Real, int DIM>
__device__ __forceinline__ void window_height_regs(GroupFixed<Real> *fx, const StepRec<Real> &st, const float4 *ca,
                                                   const float4 *cb, long long step, const DepositLog &log) {
  const bool wt = fx->wd.method != ABP_METHOD_MABP;  // mABP hills: fixed height w
  double t[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    t[c] = 0;
    if (c < (1 << DIM) && wt) {
      double w = 1;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const double f = (double)st.f[k];
        w *= ((c >> k) & 1) ? f : 1.0 - f;
      }
      double v[4];
      rec_vals<Real, DIM>(ca[c], cb[c], v);
      t[c] = w * v[0];
    }
  }
  window_height_out<Real>(fx, st, t, step, log);
}

// a2 of a window deposit, reading the corners from the grid.
template <typename Real, int DIM>
__device__ void window_height(GroupFixed<Real> *fx, const StepRec<Real> &st, long long step, const DepositLog &log) {
  float4 ca[1 << DIM], cb[1 << DIM];
  if (fx->wd.method != ABP_METHOD_MABP) interp_load<Real, DIM>(fx->wd, st, ca, cb);
  window_height_regs<Real, DIM>(fx, st, ca, cb, step, log);
}

// The deposit's axis state into the group's fixed state (threads k < d), for
// build_tables and the stencil.
template <typename Real>
__device__ __forceinline__ void window_dep_axis(const Grp &g, GroupFixed<Real> *fx, const StepRec<Real> &st) {
  if (g.t < fx->wd.g.d) {
    const int k = g.t;
    fx->da[k] = st.da[k];
    fx->dc[k] = st.dc[k];
    fx->df[k] = st.df[k];
  }
}

// The step's flags and clamp mask from its CV tasks.
template <typename Real>
__device__ __forceinline__ void step_flags(int d, bool dep, StepRec<Real> &st) {
  int flags = dep ? ABP_WFLAG_DEPOSIT : 0, clamped = 0;
  for (int k = 0; k < d; ++k) {
    flags |= st.cfl[k] & 0xffff;
    clamped |= ((st.cfl[k] >> 16) & 1) << k;
  }
  if (clamped) flags |= ABP_WFLAG_OOR;
  st.clamped = clamped;
  st.flags = flags;
}

// Per atom, its a5 terms in the order they are added (CV by CV, list A
// before list B): COM distance list A w_i, list B -w_i (both on the unit
// separation); dihedral or RMSD atom i: -1 on its gradient row.
template <typename Real>
__device__ void build_atom_terms(const Grp &g, const GroupFixed<Real> *fx, int *cnt, AtomTerm<Real> *terms) {
  const WalkerDev &wd = fx->wd;
  for (int a = g.t; a < wd.natoms; a += g.G) cnt[a] = 0;
  g.sync();
  if (g.t == 0) {
    for (int k = 0; k < wd.g.d; ++k) {
      const CvDev &c = wd.cv[k];
      const bool com = c.type == ABP_CV_COM_DIST;
      for (int l = 0; l < (com ? 2 : 1); ++l) {
        const int n = l ? c.nb : (c.type == ABP_CV_DIHEDRAL ? 4 : c.na);
        const int32_t *list = l ? fx->ib[k] : fx->ia[k];
        for (int i = 0; i < n; ++i) {
          const int at = list[i];
          AtomTerm<Real> t;
          t.w = com ? (l ? -fx->wb[k][i] : fx->wa[k][i]) : (Real)-1;
          t.off = k * 12 + (com ? 0 : 3 * i);
          terms[at * kAtomTerms + cnt[at]] = t;
          cnt[at] += 1;
        }
      }
    }
  }
  g.sync();
}

// a5 of atom a at one interpolated step, summed in the atom's term order.
template <typename Real>
__device__ __forceinline__ typename Rec4<Real>::T atom_force(const int *cnt, const AtomTerm<Real> *terms, int a,
                                                             const StepRec<Real> &st) {
  const AtomTerm<Real> *t = terms + a * kAtomTerms;
  const int ne = cnt[a];
  const Real *J = &st.jac[0][0];
  Real f0 = 0, f1 = 0, f2 = 0;
  for (int q = 0; q < ne; ++q) {
    const Real w = t[q].w;
    const Real *v = J + t[q].off;
    f0 += w * v[0];
    f1 += w * v[1];
    f2 += w * v[2];
  }
  return make_rec<Real>(f0, f1, f2, 0);
}

// Force store of the windowed form: written once and not read again here,
// so it streams past L2 (evict-first).
template <typename Real>
__device__ __forceinline__ void store_force_stream(typename Rec4<Real>::T *fo, const typename Rec4<Real>::T &f,
                                                   int mode);
template <>
__device__ __forceinline__ void store_force_stream<float>(float4 *fo, const float4 &f, int mode) {
  if (mode == ABP_FORCES_ACCUMULATE) {
    float4 o = __ldcs(fo);
    __stcs(fo, make_float4(o.x + f.x, o.y + f.y, o.z + f.z, o.w));
  } else {
    __stcs(fo, make_float4(f.x, f.y, f.z, 0.f));
  }
}
template <>
__device__ __forceinline__ void store_force_stream<double>(D4 *fo, const D4 &f, int mode) {
  double2 *p = reinterpret_cast<double2 *>(fo);
  if (mode == ABP_FORCES_ACCUMULATE) {
    double2 a = __ldcs(p), b = __ldcs(p + 1);
    __stcs(p, make_double2(a.x + f.x, a.y + f.y));
    __stcs(p + 1, make_double2(b.x + f.z, b.y));
  } else {
    __stcs(p, make_double2(f.x, f.y));
    __stcs(p + 1, make_double2(f.z, 0.0));
  }
}

}  // namespace abp
