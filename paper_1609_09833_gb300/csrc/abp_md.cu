// abp_md.cu -- the closed-loop form (abp_md_run): the force call inside a
// model MD engine on the device, so that the coordinates of step t + 1 come
// from the bias force of step t without a host round trip (the biased MD
// cycle of the paper's Figure "cycle", with overdamped Langevin dynamics in
// place of GROMACS).
//
//   k_md   four warps per walker, for walkers whose CVs are COM distances,
//          dihedrals or RMSDs (the windowed form's walkers). A step is a
//          dependent chain -- a1, a2 + a3 on deposit steps, a4, a5, the move --
//          so a walker's steps cannot overlap one another; the group keeps
//          the walker's atoms in shared memory for the whole launch, splits
//          each step's independent work between the two warps of its step
//          pair (the COM sums beside the other CVs, one atom per thread for
//          the forces and the move), draws the noise a window of steps ahead
//          on its two other warps, and runs each phase with the windowed
//          form's per-step operations (abp_window_ops.cuh): the same axis
//          state, height, stencil and interpolation arithmetic.
#include <cuda_runtime.h>

#include "abp_launch.h"
#include "abp_md.cuh"
#include "abp_window_ops.cuh"

namespace abp {

namespace {

template <typename Real>
__host__ __device__ constexpr int md_fixed_bytes() {
  return (int)((sizeof(GroupFixed<Real>) + 31) & ~(size_t)31);
}

// Steps per noise window of the closed-loop form: the producer warps fill
// one window's noise while the step chain consumes the previous one; two
// windows of a walker's noise take at most ~32 KB of shared memory.
__host__ __device__ inline int md_window(int natoms, int real) {
  int W = (32 * 1024) / (2 * natoms * 3 * real);
  return W < 1 ? 1 : (W > 16 ? 16 : W);
}

// Shared-memory layout of one walker's group (bytes from the end of its
// GroupFixed): the atoms, the step's record, the potential's gradient, two
// windows of noise, the a5 term tables and the CV atom lists.
struct MdLayout {
  int xs, st, ju, nz, nzwin, cnt, terms, lists, total, W;
};

__host__ __device__ inline MdLayout md_layout(int natoms, const CvDev *cv, int d, int fp64) {
  MdLayout L;
  const int rsz = fp64 ? 32 : 16, real = fp64 ? 8 : 4;
  L.W = md_window(natoms, real);
  int off = 0;
  L.xs = off;
  off += natoms * rsz;
  L.st = off;
  off += align32(fp64 ? (int)sizeof(StepRec<double>) : (int)sizeof(StepRec<float>));
  L.ju = off;
  off += align32(kMaxCv * 12 * real);
  L.nz = off;
  L.nzwin = align16(L.W * natoms * 3 * real);
  off += 2 * L.nzwin;
  L.cnt = off;
  off += align16(natoms * 4);
  L.terms = off;
  off += natoms * kAtomTerms * (fp64 ? 16 : 8);
  L.lists = off;
  for (int k = 0; k < d; ++k) {
    off += align16((cv[k].na + cv[k].nb) * 4);
    if (cv[k].type == ABP_CV_COM_DIST) off += align16((cv[k].na + cv[k].nb) * real);
  }
  L.total = align32(off);
  return L;
}

// One weighted offset w (p - p0) added to a lane's COM sum (FP32: Kahan).
template <typename Real>
__device__ __forceinline__ void com_term(Real w, const typename Rec4<Real>::T &p, const typename Rec4<Real>::T &p0,
                                         Real *h, Real *l) {
  const Real d[3] = {sub_rn(p.x, p0.x), sub_rn(p.y, p0.y), sub_rn(p.z, p0.z)};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if constexpr (sizeof(Real) == 4) {
      const Real y = fma_rn(w, d[q], -l[q]);
      const Real t = add_rn(h[q], y);
      l[q] = sub_rn(sub_rn(t, h[q]), y);
      h[q] = t;
    } else {
      h[q] = fma_rn(w, d[q], h[q]);
    }
  }
}

// The half-warps' sums of a COM distance combined and finished (com_warp).
template <typename Real>
__device__ __forceinline__ int com_warp_end(const CvDev &c, const typename Rec4<Real>::T &p0, Real *h, Real *l,
                                            int lane, Real &s, Real &sl, Real *u) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if constexpr (sizeof(Real) == 4) {
      // Kahan's compensation holds minus the lost part. Each level adds the
      // partner's pair as s = h + oh with its exact error (two_sum) going to
      // the low part, left unnormalised: the high parts' chain is one add
      // per level, and both partners form the same bits (a + b and the
      // exact error of a + b do not depend on the order)
      l[q] = -l[q];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const Real oh = __shfl_xor_sync(0xffffffffu, h[q], o), ol = __shfl_xor_sync(0xffffffffu, l[q], o);
        Real sq, eq;
        two_sum<Real>(h[q], oh, sq, eq);
        h[q] = sq;
        l[q] = add_rn(add_rn(l[q], ol), eq);
      }
    } else {
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) h[q] += __shfl_xor_sync(0xffffffffu, h[q], o);
    }
  }
  Real bh[3], bl[3], b0[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    bh[q] = __shfl_sync(0xffffffffu, h[q], 16);
    bl[q] = __shfl_sync(0xffffffffu, l[q], 16);
  }
  b0[0] = __shfl_sync(0xffffffffu, p0.x, 16);
  b0[1] = __shfl_sync(0xffffffffu, p0.y, 16);
  b0[2] = __shfl_sync(0xffffffffu, p0.z, 16);
  if (lane != 0) return 0;
  const Real a0[3] = {p0.x, p0.y, p0.z};
  return com_finish<Real>(c, a0, h, l, b0, bh, bl, s, sl, u);
}

// A COM distance by one warp: group A's atoms on lanes 0-15 and group B's on
// lanes 16-31 (stride 16), each lane's weighted offsets from its group's
// first atom summed (FP32: compensated, as com_sum), the half-warps' partial
// sums combined by a butterfly (FP32: in hi + lo, the low parts unnormalised),
// then finished on lane 0 (com_finish). Every lane of the warp calls it;
// lane 0 returns the CV.
template <typename Real>
__device__ __forceinline__ int com_warp(const CvDev &c, const int32_t *ia, const int32_t *ib, const Real *wa,
                                        const Real *wb, const typename Rec4<Real>::T *x, int lane, Real &s, Real &sl,
                                        Real *u) {
  const bool gb = lane >= 16;
  const int32_t *list = gb ? ib : ia;
  const Real *wts = gb ? wb : wa;
  const int n = gb ? c.nb : c.na;
  const auto p0 = x[list[0]];
  Real h[3] = {0, 0, 0}, l[3] = {0, 0, 0};
  for (int i = lane & 15; i < n; i += 16) com_term<Real>(wts[i], x[list[i]], p0, h, l);
  return com_warp_end<Real>(c, p0, h, l, lane, s, sl, u);
}

// com_warp for groups of at most 16 atoms, the lane's atom (or -1), its
// weight and its group's first atom held in registers across the launch.
template <typename Real>
__device__ __forceinline__ int com_warp_reg(const CvDev &c, int first, int atom, Real w,
                                            const typename Rec4<Real>::T *x, int lane, Real &s, Real &sl, Real *u) {
  const auto p0 = x[first];
  Real h[3] = {0, 0, 0}, l[3] = {0, 0, 0};
  if (atom >= 0) com_term<Real>(w, x[atom], p0, h, l);
  return com_warp_end<Real>(c, p0, h, l, lane, s, sl, u);
}

// The end of a4 in the closed-loop form: V and dV/ds_k (mABP: the nearest
// node's histograms turned into the bias; zero on a clamped axis; plus the
// CV range wall) into the step's record. The Jacobian factors stay unscaled:
// the force phase weighs them by dV/ds_k + dU/ds_k.
template <typename Real>
__device__ __forceinline__ void md_finish(const WalkerDev &wd, StepRec<Real> &st, Real *acc) {
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
    if (k < d) st.dv[k] = (((st.clamped >> k) & 1) ? (Real)0 : acc[1 + k]) + wall_grad<Real>(wd, k, st.s[k]);
}

// a4 by the warp: lane c < 2^DIM reads corner c and weighs its fields, the
// corners are summed by a butterfly ((c0 + c1) + (c2 + c3), ...), and lane 0
// finishes the look-up (md_finish). Every lane of the warp calls it.
template <typename Real, int DIM>
__device__ __forceinline__ void interp_warp(const WalkerDev &wd, StepRec<Real> &st, int lane) {
  constexpr int NC = 1 << DIM;
  Real acc[4] = {0, 0, 0, 0};
  if (lane < NC) {
    float4 ra, rb;
    rec_load<DIM>(node_ptr<DIM>(wd.g, corner_node<Real, DIM>(wd.g, st, lane)), ra, rb);
    Real v[4];
    rec_vals<Real, DIM>(ra, rb, v);
    const Real wc = corner_weight<Real, DIM>(st, lane);
#pragma unroll
    for (int q = 0; q <= DIM; ++q) acc[q] = wc * v[q];
  }
#pragma unroll
  for (int o = 1; o < NC; o <<= 1)
#pragma unroll
    for (int q = 0; q <= DIM; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (lane == 0) md_finish<Real>(wd, st, acc);
}

// The register-fed form's a4 (WT walkers): the grid's record pointer and
// sizes, the wall's constants in registers; the corner weights and the
// combination as interp_warp's, the clamp bits read from the CV records.
struct GridC {
  const unsigned char *rec;
  int n0, n1;
};

template <typename Real, int DIM>
__device__ __forceinline__ void interp_warp_reg(const WalkerDev &wd, const GridC &gc, Real kwall, const Real *smax,
                                                StepRec<Real> &st, int lane) {
  constexpr int NC = 1 << DIM;
  Real acc[4] = {0, 0, 0, 0};
  if (lane < NC) {
    long long node = (lane & 1) ? st.i1[0] : st.i0[0];
    if (DIM > 1) node += (long long)gc.n0 * ((lane & 2) ? st.i1[DIM > 1 ? 1 : 0] : st.i0[DIM > 1 ? 1 : 0]);
    if (DIM > 2)
      node += (long long)gc.n0 * gc.n1 * ((lane & 4) ? st.i1[DIM > 2 ? 2 : 0] : st.i0[DIM > 2 ? 2 : 0]);
    float4 ra, rb;
    rec_load<DIM>(gc.rec + chk_node(wd.g, node) * (DIM > 1 ? 32 : 16), ra, rb);
    Real v[4];
    rec_vals<Real, DIM>(ra, rb, v);
    const Real wc = corner_weight<Real, DIM>(st, lane);
#pragma unroll
    for (int q = 0; q <= DIM; ++q) acc[q] = wc * v[q];
  }
#pragma unroll
  for (int o = 1; o < NC; o <<= 1)
#pragma unroll
    for (int q = 0; q <= DIM; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  if (lane == 0) {
    st.V = acc[0];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const Real sk = st.s[k];
      const Real wall = (kwall > (Real)0 && sk > smax[k]) ? kwall * (sk - smax[k]) : (Real)0;
      st.dv[k] = (((st.cfl[k] >> 16) & 1) ? (Real)0 : acc[1 + k]) + wall;
    }
  }
}

// The step record's CV k on a step that deposits nothing (register-fed
// form): the value and the interpolation state (axis_interp_ff).
__device__ __forceinline__ void cv_rec_reg(const AxisC<float> &c, int k, float sk, float slk, int fl,
                                           StepRec<float> &st) {
  st.s[k] = sk;
  st.sl[k] = slk;
  const AxisSt<float> ax = axis_interp_ff(c, sk, slk);
  st.i0[k] = ax.i0;
  st.i1[k] = ax.i1;
  st.f[k] = ax.f;
  st.cfl[k] = fl | (ax.clamped << 16);
}

// L1 prefetch of the grid records around a cell (lower corner c0 on axis 0,
// c1 on axis 1): m0 nodes either side along axis 0, m1 rows either side
// along axis 1 (wrapped on a periodic axis, limited on the others), one
// 128-byte line per lane and request; lanes first..31 take part.
template <int DIM>
__device__ __forceinline__ void prefetch_cell(const GridDev &gd, int c0, int c1, int lane, int first) {
  if (DIM > 2 || lane < first) return;
  constexpr int rb = DIM > 1 ? 32 : 16;
  const int m0 = 4, m1 = DIM > 1 ? 8 : 0;
  int lo0 = c0 - m0, hi0 = c0 + 1 + m0;
  lo0 = lo0 < 0 ? 0 : lo0;
  hi0 = hi0 > gd.n[0] - 1 ? gd.n[0] - 1 : hi0;
  const int lines = ((hi0 * rb) >> 7) - ((lo0 * rb) >> 7) + 1;
  const int rows = 2 * m1 + 2;
  const unsigned char *rec = reinterpret_cast<const unsigned char *>(gd.rec);
  for (int r = lane - first; r < lines * rows; r += 32 - first) {
    const int row = r / lines, ln = r - row * lines;
    int j1 = 0;
    if (DIM > 1) {
      j1 = c1 - m1 + row;
      if (gd.periodic[1]) {
        if (j1 < 0) j1 += gd.n[1];
        if (j1 >= gd.n[1]) j1 -= gd.n[1];
      } else if (j1 < 0 || j1 >= gd.n[1]) {
        continue;
      }
    }
    const unsigned char *p = rec + ((long long)j1 * gd.n[0]) * rb + ((((lo0 * rb) >> 7) + ln) << 7);
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
  }
}

// a2 + a3 of a deposit step by the step pair (its own function: rarely run,
// kept out of the step loop's code): the axis state of the deposit, the
// tables, the height from the grid before the deposit, the stencil.
template <typename Real, int DIM, int UNR>
__device__ __noinline__ void md_deposit(const Grp &g, GroupFixed<Real> *fx, const StepRec<Real> &st, long long step,
                                        const DepositLog &log) {
  const GroupLayout Lnone{};
  window_dep_axis<Real>(g, fx, st);
  g.sync();
  build_tables<Real>(g, fx);
  if (g.t == 0) window_height<Real, DIM>(fx, st, step, log);
  g.sync();
  deposit_stencil<Real, false, UNR>(g, fx, Lnone, nullptr);
  g.sync();
}

// The closed-loop kernel: a group of four warps per walker.
//   warps 0 and 1, the step pair: each step's chain. Warp 0 evaluates the COM
//   distances (com_warp) and a4 (interp_warp); warp 1 evaluates the other
//   CVs (one lane per CV) beside warp 0's sums and the CV potential's
//   gradient beside a4; both run a deposit's stencil and the forces and
//   moves of the atoms. FAST (the register-fed form, chosen on the host for
//   walkers that fit it): the chain's loop invariants in registers, the
//   interpolation state of a step without a deposit by selects, the step's
//   flags on warp 1 beside a4 -- the same operations on the same values.
//   Named barrier gid + 1 (64 threads) separates the step's phases.
//   warps 2 and 3, the producers: the Philox noise of the next window of W
//   steps while the pair runs the current one (two noise buffers); then,
//   until the pair ends the window, warp 2 prefetches the grid records
//   around the walker's current cell into L1, so that a4's corner loads
//   hit there; the four warps meet at window boundaries (named barrier
//   gpc + gid + 1). A step's finiteness check is made on the coordinates as
//   the move writes them (the launch's first ones before the first step).
template <typename Real, int DIM, int UNR, bool FAST>
__global__ void __launch_bounds__(256, 1) k_md(MdRunArgs a) {
  using R4 = typename Rec4<Real>::T;
  extern __shared__ __align__(32) unsigned char smem[];
  const RunArgs &ra = a.r;
  const int gpc = blockDim.x >> 7;  // walker groups per CTA
  const int gid = threadIdx.x >> 7;
  const int slot = blockIdx.x * gpc + gid;
  if (slot >= ra.nw) return;  // the whole group
  const int tg = threadIdx.x & 127;
  Grp gg;  // the whole group
  gg.G = 128;
  gg.gid = gpc + gid;
  gg.t = tg;
  gg.lane = tg & 31;
  gg.warp = tg >> 5;
  gg.nwarps = 4;
  // the step pair's barrier: bar.sync itself makes the participating
  // threads' earlier shared and global accesses visible to one another
  auto psync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(64) : "memory"); };
  Grp g;  // the step pair (warps 0, 1) or the producer pair (warps 2, 3)
  g.G = 64;
  g.gid = gid;
  g.t = tg & 63;
  g.lane = tg & 31;
  g.warp = g.t >> 5;
  g.nwarps = 2;
  const bool producer = tg >= 64;
  const bool w0 = !producer && g.warp == 0;
  const int lane = g.lane;
  unsigned char *base = smem + (size_t)gid * ra.group_bytes;
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(base);
  unsigned char *dyn = base + md_fixed_bytes<Real>();
  const TableEntry te = ra.table[slot];
  // The launch's global reads go out in one wave: the descriptor's copy, and
  // beside it (read from the global descriptor itself) the CV atom lists and
  // COM weights, the a5 term tables and the atoms.
  const WalkerDev *gw = te.wd;
  {
    const int *s = reinterpret_cast<const int *>(gw);
    int *d = reinterpret_cast<int *>(&fx->wd);
    for (int i = tg; i < (int)(sizeof(WalkerDev) / 4); i += 128) d[i] = s[i];
  }
  const int natoms = gw->natoms;
  const MdLayout L = md_layout(natoms, gw->cv, DIM, sizeof(Real) == 8);
  {
    // the CV atom lists (and COM weights) into shared memory
    unsigned char *cur = dyn + L.lists;
    for (int k = 0; k < DIM; ++k) {
      const CvDev &c = gw->cv[k];
      int32_t *ia = reinterpret_cast<int32_t *>(cur);
      int32_t *ib = ia + c.na;
      for (int i = tg; i < c.na; i += 128) ia[i] = c.ia[i];
      for (int i = tg; i < c.nb; i += 128) ib[i] = c.ib[i];
      cur += align16((c.na + c.nb) * 4);
      Real *w_a = nullptr, *w_b = nullptr;
      if (c.type == ABP_CV_COM_DIST) {
        w_a = reinterpret_cast<Real *>(cur);
        w_b = w_a + c.na;
        for (int i = tg; i < c.na; i += 128) w_a[i] = sizeof(Real) == 4 ? (Real)c.wa[i] : (Real)c.wa64[i];
        for (int i = tg; i < c.nb; i += 128) w_b[i] = sizeof(Real) == 4 ? (Real)c.wb[i] : (Real)c.wb64[i];
        cur += align16((c.na + c.nb) * (int)sizeof(Real));
      }
      if (tg == 0) {
        fx->ia[k] = ia;
        fx->ib[k] = ib;
        fx->wa[k] = w_a;
        fx->wb[k] = w_b;
      }
    }
  }
  R4 *xs = reinterpret_cast<R4 *>(dyn + L.xs);
  StepRec<Real> &st = *reinterpret_cast<StepRec<Real> *>(dyn + L.st);
  int *cnt = reinterpret_cast<int *>(dyn + L.cnt);
  AtomTerm<Real> *terms = reinterpret_cast<AtomTerm<Real> *>(dyn + L.terms);
  const bool tables = gw->acnt != nullptr;  // the a5 term tables built at walker creation
  if (tables) {
    const AtomTerm<Real> *gt = reinterpret_cast<const AtomTerm<Real> *>(gw->aterms);
    for (int i = tg; i < natoms; i += 128) cnt[i] = gw->acnt[i];
    for (int i = tg; i < natoms * kAtomTerms; i += 128) terms[i] = gt[i];
  }
  R4 *cio = reinterpret_cast<R4 *>(const_cast<void *>(ra.coords)) + ra.coff[te.idx];
  for (int i = tg; i < natoms; i += 128) xs[i] = cio[i];
  gg.sync();
  const WalkerDev &wd = fx->wd;
  if (!tables && !producer) build_atom_terms<Real>(g, fx, cnt, terms);
  R4 *fout = ra.forces ? reinterpret_cast<R4 *>(ra.forces) + ra.foff[te.idx] : reinterpret_cast<R4 *>(wd.fbuf);
  const int fmode = ra.forces ? ra.mode : ABP_FORCES_OVERWRITE;
  R4 *tout = a.traj ? reinterpret_cast<R4 *>(a.traj) + a.toff[te.idx] : nullptr;
  const long long step0 = ra.step0;
  const MdCoef<Real> mc = md_coef<Real>(a.md);
  const MdTerm<Real> mt = md_term<Real>(a.md, lane);
  const int W = L.W, nwin = (ra.nsteps + W - 1) / W;
  auto nzbuf = [&](int w) { return reinterpret_cast<Real *>(dyn + L.nz + (w & 1) * L.nzwin); };
  // the producers: window w's noise, (step, atom) pairs over their 64 threads
  auto draw = [&](int w) {
    Real *nz = nzbuf(w);
    const int t0 = w * W, nt = min(W, ra.nsteps - t0);
    for (Iter2 it(g.t, 64, natoms); it.j < nt; it.next()) {
      Real n3[3];
      md_normals(a.md.seed, te.stream, step0 + t0 + it.j, it.i, n3);
      Real *p = nz + (it.j * natoms + it.i) * 3;
      p[0] = n3[0];
      p[1] = n3[1];
      p[2] = n3[2];
    }
  };
  long long rem = step0 % wd.stride;
  long long next_dep = rem == 0 ? 0 : wd.stride - rem;
  int last = -1;        // the last step run
  bool stopped = false;  // non-finite coordinates met (the pair's decision)
  Real *dUs = reinterpret_cast<Real *>(dyn + L.ju);  // the step's dU/ds_k (warp 1 -> the force phase)
  // [0], [1]: non-finite coordinates seen by each step-pair warp; [2]: the
  // number of windows the pair has finished (the producers' prefetch stops)
  int *badw = reinterpret_cast<int *>(fx->winbad);
  if (tg == 0) badw[2] = 0;
  if (producer && nwin > 0) draw(0);
  if (!producer) {
    // the launch's first coordinates; later steps' are checked as they are made
    int bad = 0;
    for (int i = g.t; i < natoms; i += 64) bad |= finite_rec<Real>(xs[i]) ? 0 : 1;
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) badw[g.warp] = bad;
  }
  gg.sync();
  // FAST (every walker of the launch has COM groups of at most 16 atoms,
  // dihedrals as its other CVs, and at most 64 atoms of at most two a5
  // terms each): the step chain's loop invariants in registers -- the
  // lane's COM atom, weight and group head, the dihedral lane's four atoms,
  // the thread's atom's a5 terms
  unsigned com_mask = 0;  // bit k: CV k is a COM distance
#pragma unroll
  for (int k = 0; k < DIM; ++k) com_mask |= (wd.cv[k].type == ABP_CV_COM_DIST ? 1u : 0u) << k;
  int cfirst[DIM], catom[DIM], datom[4] = {0, 0, 0, 0};
  Real cw[DIM];
  int tne = 0, to0 = 0, to1 = 0, tk0 = 0, tk1 = 0;
  Real tw0 = 0, tw1 = 0;
  AxisC<Real> axc[DIM];
  GridC gc{nullptr, 0, 0};
  Real kwall = 0, smax[DIM];
  if (FAST && !producer) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      axc[k] = axis_consts<Real>(wd.g, k);
      smax[k] = wd.smax_f[k];
    }
    kwall = wd.kwall_f;
    gc.rec = reinterpret_cast<const unsigned char *>(wd.g.rec);
    gc.n0 = wd.g.n[0];
    gc.n1 = DIM > 1 ? wd.g.n[DIM > 1 ? 1 : 0] : 0;
    int q = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      cfirst[k] = catom[k] = 0;
      cw[k] = 0;
      if ((com_mask >> k) & 1) {
        const bool gb = lane >= 16;
        const int n = gb ? wd.cv[k].nb : wd.cv[k].na;
        const int32_t *list = gb ? fx->ib[k] : fx->ia[k];
        const Real *wts = gb ? fx->wb[k] : fx->wa[k];
        cfirst[k] = list[0];
        if ((lane & 15) < n) {
          catom[k] = list[lane & 15];
          cw[k] = wts[lane & 15];
        } else {
          catom[k] = -1;
        }
      } else {
        if (lane == q)
#pragma unroll
          for (int j = 0; j < 4; ++j) datom[j] = fx->ia[k][j];
        ++q;
      }
    }
    if (g.t < natoms) {
      const AtomTerm<Real> *ti = terms + g.t * kAtomTerms;
      tne = cnt[g.t];
      if (tne > 0) {
        to0 = ti[0].off;
        tw0 = ti[0].w;
        tk0 = to0 >= 24 ? 2 : (to0 >= 12 ? 1 : 0);
      }
      if (tne > 1) {
        to1 = ti[1].off;
        tw1 = ti[1].w;
        tk1 = to1 >= 24 ? 2 : (to1 >= 12 ? 1 : 0);
      }
    }
  }
  for (int w = 0; w < nwin; ++w) {
    if (producer) {
      if (w + 1 < nwin) draw(w + 1);
      if (DIM <= 2 && g.warp == 0) {
        // until the pair ends the window: L1 prefetch around the walker's
        // current cell (read while the pair may be writing it; clamped to
        // the grid), bounded
        const volatile int *vdone = badw + 2;
        const volatile int *vi0 = reinterpret_cast<const volatile int *>(st.i0);
        int l0 = -1, l1 = -1;
        for (int it = 0; it < (1 << 16) && *vdone != w + 1; ++it) {
          int c0 = vi0[0], c1 = DIM > 1 ? vi0[DIM > 1 ? 1 : 0] : 0;
          c0 = c0 < 0 ? 0 : (c0 > wd.g.n[0] - 1 ? wd.g.n[0] - 1 : c0);
          if (DIM > 1) c1 = c1 < 0 ? 0 : (c1 > wd.g.n[DIM > 1 ? 1 : 0] - 1 ? wd.g.n[DIM > 1 ? 1 : 0] - 1 : c1);
          if (c0 != l0 || c1 != l1) {
            prefetch_cell<DIM>(wd.g, c0, c1, lane, 0);
            l0 = c0;
            l1 = c1;
          }
          __nanosleep(200);
        }
      }
    } else {
      const Real *nzw = nzbuf(w);
      const int t0 = w * W, nt = min(W, ra.nsteps - t0);
      for (int j = 0; j < nt && !stopped; ++j) {
        const int t = t0 + j;
        const long long step = step0 + t;
        const bool dep = t == next_dep;
        if (dep) next_dep += wd.stride;
        if (badw[0] | badw[1]) {
          // this walker stops here: its state says so, its atoms stay
          if (g.t == 0) {
            wd.state->flags = ABP_WFLAG_NONFINITE;
            atomicAdd(&ra.ctr->nonfinite, 1);
          }
          stopped = true;
          break;
        }
        // a1
        if (w0) {
#pragma unroll
          for (int k = 0; k < DIM; ++k)
            if ((com_mask >> k) & 1) {
              Real sk, slk;
              const int fl =
                  FAST ? com_warp_reg<Real>(wd.cv[k], cfirst[k], catom[k], cw[k], xs, lane, sk, slk, st.jac[k])
                       : com_warp<Real>(wd.cv[k], fx->ia[k], fx->ib[k], fx->wa[k], fx->wb[k], xs, lane, sk, slk,
                                        st.jac[k]);
              if (lane == 0) {
                if constexpr (FAST) {
                  if (!dep) {
                    cv_rec_reg(axc[k], k, sk, slk, fl, st);
                    continue;
                  }
                }
                window_cv_rec<Real>(wd, k, sk, slk, fl, dep, st);
              }
            }
        } else {
          int q = 0;
#pragma unroll
          for (int k = 0; k < DIM; ++k)
            if (!((com_mask >> k) & 1)) {
              if (lane == q) {
                if constexpr (FAST) {
                  Real x4[4][3];
#pragma unroll
                  for (int j = 0; j < 4; ++j) {
                    const R4 p = xs[datom[j]];
                    x4[j][0] = p.x;
                    x4[j][1] = p.y;
                    x4[j][2] = p.z;
                  }
                  Real sk, slk;
                  const int fl = dihedral_core<Real>(wd.cv[k], x4, sk, reinterpret_cast<Real(*)[3]>(st.jac[k]), slk);
                  if constexpr (FAST) {
                    if (dep)
                      window_cv_rec<Real>(wd, k, sk, slk, fl, dep, st);
                    else
                      cv_rec_reg(axc[k], k, sk, slk, fl, st);
                  }
                } else {
                  window_cv<Real>(fx, xs, k, dep, st);
                }
              }
              ++q;
            }
        }
        psync();
        // the step's flags (read after the launch): by warp 0 ahead of a4, or
        // in the register-fed form by warp 1 beside it
        if (!FAST && w0 && lane == 0) step_flags<Real>(DIM, dep, st);
        if (dep) {
          psync();
          md_deposit<Real, DIM, UNR>(g, fx, st, step, ra.log);
        }
        if (w0) {
          // a4 by warp 0
          if (FAST)
            interp_warp_reg<Real, DIM>(wd, gc, kwall, smax, st, lane);
          else
            interp_warp<Real, DIM>(wd, st, lane);
        } else {
          // beside it, the CV potential's gradient by warp 1
          Real sk[3] = {0, 0, 0}, dU[3];
#pragma unroll
          for (int k = 0; k < DIM; ++k) sk[k] = st.s[k];
          md_potential_grad_warp<Real>(mc, mt, sk, lane, dU);
          if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) dUs[k] = dU[k];
            if (FAST) step_flags<Real>(DIM, dep, st);
          }
        }
        psync();
        // a5 and the move, one atom per thread of the pair: each of the
        // atom's terms (CV k, weight w, Jacobian factor v) adds w v (dV_b/ds_k
        // + dU/ds_k) to the total force, and w v dV_b/ds_k to the bias force
        // when the caller keeps it; then x += c1 F + c2 xi
        const Real *nz = nzw + j * natoms * 3;
        const bool keep_f = ra.forces || t == ra.nsteps - 1;
        Real dvk[3], dtk[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          dvk[k] = k < DIM ? st.dv[k] : (Real)0;
          dtk[k] = dvk[k] + dUs[k];
        }
        const Real *J = &st.jac[0][0];
        // atom i's force from its terms' sums f (total) and b (bias), the
        // bias force to the caller, the move
        auto move = [&](int i, const Real *f, const Real *b) {
          R4 x = xs[i];
          if (tout) tout[(long long)t * a.tstride + i] = x;
          if (keep_f) {
            R4 *fo = fout + (ra.forces ? (long long)t * ra.fstride : 0) + i;
            store_force<Real>(fo, make_rec<Real>(b[0], b[1], b[2], 0), fmode);
          }
          x.x = add_rn(x.x, fma_rn(mc.c1, f[0], mul_rn(mc.c2, nz[3 * i])));
          x.y = add_rn(x.y, fma_rn(mc.c1, f[1], mul_rn(mc.c2, nz[3 * i + 1])));
          x.z = add_rn(x.z, fma_rn(mc.c1, f[2], mul_rn(mc.c2, nz[3 * i + 2])));
          xs[i] = x;
          return finite_rec<Real>(x) ? 0 : 1;
        };
        // one term: CV k's Jacobian row v of weight w
        auto term = [&](const Real *v, Real w, Real dt, Real dv, Real *f, Real *b) {
          const Real wt = mul_rn(w, dt);
#pragma unroll
          for (int q = 0; q < 3; ++q) f[q] = fma_rn(wt, v[q], f[q]);
          if (keep_f) {
            const Real wb = mul_rn(w, dv);
#pragma unroll
            for (int q = 0; q < 3; ++q) b[q] = fma_rn(wb, v[q], b[q]);
          }
        };
        int nbad = 0;
        if constexpr (FAST) {
          if (g.t < natoms) {
            Real f[3] = {0, 0, 0}, b[3] = {0, 0, 0};
            if (tne > 0)
              term(J + to0, tw0, tk0 == 0 ? dtk[0] : (tk0 == 1 ? dtk[1] : dtk[2]),
                   tk0 == 0 ? dvk[0] : (tk0 == 1 ? dvk[1] : dvk[2]), f, b);
            if (tne > 1)
              term(J + to1, tw1, tk1 == 0 ? dtk[0] : (tk1 == 1 ? dtk[1] : dtk[2]),
                   tk1 == 0 ? dvk[0] : (tk1 == 1 ? dvk[1] : dvk[2]), f, b);
            nbad = move(g.t, f, b);
          }
        } else {
          for (int i = g.t; i < natoms; i += 64) {
            const AtomTerm<Real> *ti = terms + i * kAtomTerms;
            const int ne = cnt[i];
            Real f[3] = {0, 0, 0}, b[3] = {0, 0, 0};
            for (int q = 0; q < ne; ++q) {
              const int off = ti[q].off;
              const int k = off >= 24 ? 2 : (off >= 12 ? 1 : 0);
              term(J + off, ti[q].w, dtk[k], dvk[k], f, b);
            }
            nbad |= move(i, f, b);
          }
        }
        // the next step's coordinates: each warp's half of the finiteness check
        nbad = __any_sync(0xffffffffu, nbad);
        if (lane == 0) badw[g.warp] = nbad;
        last = t;
        psync();
      }
      if (g.t == 0) *reinterpret_cast<volatile int *>(badw + 2) = w + 1;  // the pair's thread 0
    }
    gg.sync();
  }
  // the moved atoms back to the caller, and the walker's state after its
  // last step
  for (int i = tg; i < natoms; i += 128) cio[i] = xs[i];
  if (tg == 0 && last >= 0) {
    WalkerState ws;
    for (int k = 0; k < 3; ++k) {
      ws.s[k] = k < DIM ? (double)st.s[k] + (double)st.sl[k] : 0.0;
      ws.dV[k] = k < DIM ? (double)st.dv[k] : 0.0;
    }
    ws.V = (double)st.V;
    // a walker stopped by non-finite coordinates keeps its last completed
    // step's state and reports the stop
    ws.flags = stopped ? ABP_WFLAG_NONFINITE : st.flags;
    ws.pad = 0;
    ws.step = step0 + last;
    *wd.state = ws;
  }
}

}  // namespace

int md_group_bytes(const WalkerDev &hd, int fp64) {
  const int fixed = fp64 ? md_fixed_bytes<double>() : md_fixed_bytes<float>();
  return align32(fixed + md_layout(hd.natoms, hd.cv, hd.g.d, fp64).total);
}

cudaError_t launch_md(const MdRunArgs &a, int fp64, int dim, bool fast, cudaStream_t st) {
  const RunArgs &r = a.r;
  if (r.nw == 0) return cudaSuccess;
  const int gpc = r.groups_per_cta;
  const int threads = 128 * gpc;
  const int blocks = (r.nw + gpc - 1) / gpc;
  const size_t smem = (size_t)r.group_bytes * gpc;
  void (*k)(MdRunArgs);
  if (fp64)
    k = dim == 1 ? k_md<double, 1, 4, false> : dim == 2 ? k_md<double, 2, 4, false> : k_md<double, 3, 4, false>;
  else if (fast)  // four stencil nodes in flight per thread: measured best for this form's registers
    k = dim == 1 ? k_md<float, 1, 4, true> : dim == 2 ? k_md<float, 2, 4, true> : k_md<float, 3, 4, true>;
  else
    k = dim == 1 ? k_md<float, 1, 7, false> : dim == 2 ? k_md<float, 2, 7, false> : k_md<float, 3, 7, false>;
  cudaError_t e = smem_attr(reinterpret_cast<const void *>(k), smem);
  if (e != cudaSuccess) return e;
  k<<<blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace abp
