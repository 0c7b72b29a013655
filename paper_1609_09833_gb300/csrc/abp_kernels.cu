// abp_kernels.cu -- the kernels of the force call and their launchers:
//   k_run      fused batched form: one walker group per walker, steps a1..a5
//              for nsteps consecutive MD steps in one launch; the next step's
//              coordinates stream into shared memory (cp.async) while the
//              current step runs, and an optional shared-memory tile of the
//              walker's grid serves the interpolation and the deposit;
//   k_plain_*  plain form: CV, deposit and interpolation/force as separate
//              single-walker launches (the comparison point);
//   k_deliver  copies each walker's force buffer to the caller (abp_forces).
#include <cuda_runtime.h>

#include "abp_device.cuh"
#include "abp_launch.h"
#include "abp_window_ops.cuh"

namespace abp {

template <typename Real>
__host__ __device__ constexpr int fixed_bytes() {
  return (int)((sizeof(GroupFixed<Real>) + 31) & ~(size_t)31);
}

int group_fixed_bytes(int fp64) { return fp64 ? fixed_bytes<double>() : fixed_bytes<float>(); }

template <typename Real>
__device__ __forceinline__ void copy_desc(const Grp &g, WalkerDev *dst, const WalkerDev *src) {
  const int *s = reinterpret_cast<const int *>(src);
  int *d = reinterpret_cast<int *>(dst);
  for (int i = g.t; i < (int)(sizeof(WalkerDev) / 4); i += g.G) d[i] = s[i];
}

template <typename Real>
__device__ __forceinline__ GroupLayout layout_of(const GroupFixed<Real> *fx, int nwarps, int tile_budget,
                                                 bool window) {
  return group_layout(fx->wd.natoms, fx->wd.cv, fx->wd.g, fx->wd.R, nwarps, (int)sizeof(typename Rec4<Real>::T),
                      tile_budget, window, fx->wd.method == ABP_METHOD_MABP);
}

// Copy each CV's atom lists (and COM weights as Real) into shared memory and
// point fx->ia/ib/wa/wb at them. Caller syncs.
template <typename Real>
__device__ void setup_lists(const Grp &g, GroupFixed<Real> *fx, unsigned char *mem) {
  const WalkerDev &wd = fx->wd;
  unsigned char *cur = mem;
  for (int k = 0; k < wd.g.d; ++k) {
    const CvDev &c = wd.cv[k];
    int32_t *ia = reinterpret_cast<int32_t *>(cur);
    int32_t *ib = ia + c.na;
    for (int i = g.t; i < c.na; i += g.G) ia[i] = c.ia[i];
    for (int i = g.t; i < c.nb; i += g.G) ib[i] = c.ib[i];
    cur += align16((c.na + c.nb) * 4);
    Real *wa = nullptr, *wb = nullptr;
    if (c.type == ABP_CV_COM_DIST) {
      wa = reinterpret_cast<Real *>(cur);
      wb = wa + c.na;
      for (int i = g.t; i < c.na; i += g.G) wa[i] = sizeof(Real) == 4 ? (Real)c.wa[i] : (Real)c.wa64[i];
      for (int i = g.t; i < c.nb; i += g.G) wb[i] = sizeof(Real) == 4 ? (Real)c.wb[i] : (Real)c.wb64[i];
      cur += align16((c.na + c.nb) * (int)sizeof(Real));
    }
    if (g.t == 0) {
      fx->ia[k] = ia;
      fx->ib[k] = ib;
      fx->wa[k] = wa;
      fx->wb[k] = wb;
    }
  }
}

template <typename Real>
__device__ __forceinline__ unsigned char *cn_slot(unsigned char *cnmem, const WalkerDev &wd, int k, int nwarps) {
  int rsz = (int)sizeof(typename Rec4<Real>::T);
  unsigned char *cur = cnmem;
  for (int q = 0; q < k; ++q) {
    const CvDev &c = wd.cv[q];
    if (c.type == ABP_CV_COORD) cur += (c.na + c.nb) * rsz + align32(nwarps * c.na * 3 * (int)sizeof(Real));
  }
  return cur;
}

// a1 for every CV of the walker (coordinates in xs); ends with a group sync.
// CVs write disjoint state, so no sync is needed between them.
template <typename Real>
__device__ void eval_cvs(const Grp &g, GroupFixed<Real> *fx, const typename Rec4<Real>::T *xs, unsigned char *cnmem) {
  using R4 = typename Rec4<Real>::T;
  const WalkerDev &wd = fx->wd;
  for (int k = 0; k < wd.g.d; ++k) {
    const CvDev &c = wd.cv[k];
    if (c.type == ABP_CV_COM_DIST) {
      cv_com<Real>(g, fx, k, xs);
    } else if (c.type == ABP_CV_DIHEDRAL) {
      cv_dihedral<Real>(g, fx, k, xs);
    } else {
      unsigned char *slot = cn_slot<Real>(cnmem, wd, k, g.nwarps);
      R4 *jA = reinterpret_cast<R4 *>(slot);
      R4 *jB = jA + c.na;
      Real *lig = reinterpret_cast<Real *>(jB + c.nb);
      g.sync();
      cv_coord<Real>(g, fx, k, xs, jA, jB, lig);
    }
  }
  g.sync();
}

// a2 + a3: tables, height from the grid before the deposit, the stencil.
template <typename Real, bool TILE, int UNR = 4>
__device__ void deposit_step(const Grp &g, GroupFixed<Real> *fx, const GroupLayout &L, unsigned char *tile,
                             long long step, const DepositLog &log) {
  const WalkerDev &wd = fx->wd;
  build_tables<Real>(g, fx);
  if (g.warp == 0) {
    // mABP hills have the fixed height w; WT hills the well-tempered height
    const bool mabp = wd.method == ABP_METHOD_MABP;
    double V0 = mabp ? 0.0 : height_interp<Real, TILE>(fx, L, tile, g.lane);
    if (g.lane == 0) {
      double h = mabp ? wd.w : wd.w * exp(-V0 * wd.inv_dT);
      fx->hf = (Real)h;
      fx->flags |= ABP_WFLAG_DEPOSIT;
      if (log.rec) {
        unsigned long long slot = atomicAdd(log.count, 1ull);
        if (slot < log.cap) {
          abp_deposit_rec r;
          r.step = step;
          r.walker_id = wd.id;
          for (int k = 0; k < 3; ++k) {
            r.ic[k] = k < wd.g.d ? fx->ic_log[k] : 0;
            r.s[k] = k < wd.g.d ? (double)fx->sh[k] + (double)fx->sl[k] : 0.0;
          }
          r.height = h;
          log.rec[slot] = r;
        }
      }
    }
  }
  g.sync();
  deposit_stencil<Real, TILE, UNR>(g, fx, L, tile);
  g.sync();
}

template <typename Real>
__device__ void write_state(GroupFixed<Real> *fx, long long step) {
  const WalkerDev &wd = fx->wd;
  WalkerState st;
  for (int k = 0; k < 3; ++k) {
    st.s[k] = k < wd.g.d ? (double)fx->sh[k] + (double)fx->sl[k] : 0.0;
    st.dV[k] = k < wd.g.d ? (double)fx->dV[k] : 0.0;
  }
  st.V = (double)fx->V;
  st.flags = fx->flags;
  st.pad = 0;
  st.step = step;
  *wd.state = st;
}

// nsteps MD steps of one walker (steps a1..a5 each), by one group.
template <typename Real, bool TILE>
__device__ void walker_steps(const Grp &g, GroupFixed<Real> *fx, unsigned char *dyn, const GroupLayout &L,
                             const RunArgs &a, int widx) {
  using R4 = typename Rec4<Real>::T;
  const WalkerDev &wd = fx->wd;
  const int natoms = wd.natoms, d = wd.g.d;
  R4 *xb[2] = {reinterpret_cast<R4 *>(dyn + L.xs0), reinterpret_cast<R4 *>(dyn + L.xs1)};
  R4 *fs = reinterpret_cast<R4 *>(dyn + L.fs);
  unsigned char *cnmem = dyn + L.cn;
  unsigned char *tile = dyn + L.tile;
  const R4 *cin = reinterpret_cast<const R4 *>(a.coords);
  R4 *fout = a.forces ? reinterpret_cast<R4 *>(a.forces) : reinterpret_cast<R4 *>(wd.fbuf);
  const long long coff = a.coff[widx];
  const long long foff = a.forces ? a.foff[widx] : 0;
  const int mode = a.forces ? a.mode : ABP_FORCES_OVERWRITE;
  const int pieces = natoms * (int)(sizeof(R4) / 16);
  const long long step0 = a.wstep ? a.wstep[widx] : a.step0;
  auto prefetch = [&](int t, R4 *dst) {
    const unsigned char *src = reinterpret_cast<const unsigned char *>(cin + coff + (long long)t * a.cstride);
    for (int p = g.t; p < pieces; p += g.G) cp_async16(reinterpret_cast<unsigned char *>(dst) + p * 16, src + p * 16);
    cp_async_commit();
  };
  long long rem = step0 % wd.stride;
  long long next_dep = rem == 0 ? 0 : wd.stride - rem;  // step index (t) of the next deposit
  if (TILE && g.t == 0) {
    fx->reload = 1;
    for (int k = 0; k < kMaxCv; ++k) fx->org[k] = 0;
  }
  prefetch(0, xb[0]);
  for (int t = 0; t < a.nsteps; ++t) {
    const long long step = step0 + t;
    R4 *xs = xb[t & 1];
    cp_async_wait_all();
    g.sync();
    const bool dep = (t == next_dep);
    if (dep) next_dep += wd.stride;
    R4 *fo = fout + foff + (a.forces ? (long long)t * a.fstride : 0);
    int bad = 0;
    for (int i = g.t; i < natoms; i += g.G) {
      bad |= finite_rec<Real>(xs[i]) ? 0 : 1;
      fs[i] = make_rec<Real>(0, 0, 0, 0);
    }
    if (g.t == 0) {
      fx->flags = 0;
      fx->clamped = 0;
    }
    if (grp_any<Real>(g, fx, bad)) {
      // non-finite coordinates: no deposit, zero bias force, state kept
      if (t + 1 < a.nsteps) prefetch(t + 1, xb[(t + 1) & 1]);
      if (mode == ABP_FORCES_OVERWRITE)
        for (int i = g.t; i < natoms; i += g.G) fo[i] = make_rec<Real>(0, 0, 0, 0);
      if (g.t == 0) {
        wd.state->flags = ABP_WFLAG_NONFINITE;
        atomicAdd(&a.ctr->nonfinite, 1);
      }
      continue;
    }
    g.sync();
    eval_cvs<Real>(g, fx, xs, cnmem);
    // the next step's coordinates stream in while this step finishes
    if (t + 1 < a.nsteps) prefetch(t + 1, xb[(t + 1) & 1]);
    if (g.t < d) {
      axis_setup<Real>(fx, g.t, dep);
      if (TILE) tile_check_axis<Real>(fx, L, g.t, dep);
    }
    g.sync();
    if (TILE && fx->reload) {
      tile_load<Real>(g, fx, L, tile);
      if (g.t == 0) fx->reload = 0;
    }
    if (dep) deposit_step<Real, TILE>(g, fx, L, tile, step, a.log);
    interp_step<Real, TILE>(g, fx, L, tile);
    scatter_forces<Real>(g, fx, fs, cnmem);
    for (int i = g.t; i < natoms; i += g.G) store_force<Real>(fo + i, fs[i], mode);
    if (t == a.nsteps - 1 && g.t == 0) write_state<Real>(fx, step);
  }
}

// ---------------------------------------------------------------- windowed form
//
// Walkers whose CVs are all COM distances, dihedrals or RMSDs of at most 4
// atoms run their nsteps MD steps in windows of L.win steps. A window's
// coordinates arrive by cp.async two windows ahead; each window goes through
// three phases:
//   A  a1 (CVs, Jacobian factors, axis state) into the window's StepRecs,
//      one lane per (CV, step) -- two for a COM distance -- and the
//      non-finite check of every (step, atom);
//   B  the grid chain: a4 for the steps before the window's first deposit,
//      then each deposit in step order (a2 + a3) followed by a4 of the steps
//      up to the next one (windows with one deposit and a small box: one
//      round of grid reads for all of it, see chain_one);
//   C  a5 for every (step, atom) pair from the atom's list entries, summed
//      in registers in CV order and stored.
// A group's two halves run A and C, and B, on three StepRec slots (see
// walker_window). Every step reads the grid with exactly the deposits of the
// steps before it and its own: the per-step order of the method, with the
// step-independent work of a window done side by side. A step's arithmetic
// does not depend on the window it falls in or on the launch shape, so
// chunked calls and different group sizes give the same bits.

__device__ __forceinline__ float4 lds128(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts128(unsigned a, const float4 &v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

// Deposit steps of a window (bit j: step t0 + j).
__device__ __forceinline__ unsigned window_dmask(long long step0, int t0, int nt, long long stride) {
  const long long rem = (step0 + t0) % stride;
  unsigned m = 0;
  for (long long j = rem == 0 ? 0 : stride - rem; j < nt; j += stride) m |= 1u << (int)j;
  return m;
}

// Grid byte offset of node (b0 + o0, b1 + o1) of a stencil box whose first
// node is (b0, b1) (unwrapped; one wrap on a periodic axis), or -1 where it
// falls outside a non-periodic axis.
template <int DIM>
__device__ __forceinline__ long long box_node_off(const GridDev &gd, int b0, int b1, int o0, int o1, int rb) {
  int j0 = b0 + o0, j1 = b1 + o1;
  bool in = true;
  if (gd.periodic[0]) {
    if (j0 < 0) j0 += gd.n[0];
    if (j0 >= gd.n[0]) j0 -= gd.n[0];
  } else {
    in = j0 >= 0 && j0 < gd.n[0];
  }
  if (DIM > 1) {
    if (gd.periodic[1]) {
      if (j1 < 0) j1 += gd.n[1];
      if (j1 >= gd.n[1]) j1 -= gd.n[1];
    } else {
      in = in && j1 >= 0 && j1 < gd.n[1];
    }
  }
  return in ? chk_node(gd, j0 + (DIM > 1 ? (long long)gd.n[0] * j1 : 0)) * rb : -1;
}

// Named barrier `id` of `n` threads: arrive without waiting (after this
// thread's shared-memory writes), or wait for the phase to complete.
__device__ __forceinline__ void bar_arrive(int id, int n) {
  __threadfence_block();
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_wait(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Phases of one window, each run by a (sub)group `g` that ends synchronised.
template <typename Real>
struct WindowCtx {
  using R4 = typename Rec4<Real>::T;
  GroupFixed<Real> *fx;
  GroupLayout L;          // copies, so the context stays in registers
  const void *coords;
  void *out;             // the caller's force records (NULL: the walker's own buffer)
  long long cstride, fstride;
  int nsteps, xst;
  DevCounters *ctr;
  DepositLog log;
  R4 *xb[2];
  StepRec<Real> *steps;  // 3 windows of W records
  int *cnt;
  AtomTerm<Real> *terms;
  long long coff, foff, step0, last;
  int W, nwin, mode;
  bool serial_out;
  unsigned long long stream;
  unsigned char *box;    // a deposit's stencil box (WT) or the union of a window's boxes (mABP); NULL: none

  __device__ __forceinline__ int nt_of(int w) const { return min(W, nsteps - w * W); }
  __device__ __forceinline__ StepRec<Real> *steps_of(int w) const { return steps + (w % 3) * W; }

  // coordinates of window w into its buffer (one cp.async commit group)
  __device__ __forceinline__ void prefetch(const Grp &g, int w) const {
    const int t0 = w * W, nt = nt_of(w);
    const int pieces = fx->wd.natoms * (int)(sizeof(R4) / 16);
    const R4 *cin = reinterpret_cast<const R4 *>(coords);
    R4 *dst = xb[w & 1];
    for (Iter2 it(g.t, g.G, pieces); it.j < nt; it.next()) {
      const unsigned char *src =
          reinterpret_cast<const unsigned char *>(cin + coff + (long long)(t0 + it.j) * cstride) + it.i * 16;
      cp_async16_hint(reinterpret_cast<unsigned char *>(dst + it.j * xst) + it.i * 16, src, stream);
    }
    cp_async_commit();
  }

  // A: a1 and the axis state, one thread per (CV, step) -- two for a COM
  // distance, one per atom group -- and the non-finite check, on the threads
  // the tasks leave free while they run, else before them. (A step's CVs are
  // evaluated either way; those of a non-finite step are not used.)
  __device__ __forceinline__ void cvs(const Grp &g, int w) const {
    const WalkerDev &wd = fx->wd;
    const int nt = nt_of(w), natoms = wd.natoms, d = wd.g.d;
    const R4 *xs = xb[w & 1];
    StepRec<Real> *st = steps_of(w);
    unsigned *badp = &fx->winbad[w % 3];
    const unsigned dmask = window_dmask(step0, w * W, nt, wd.stride);
    // first thread of each CV's tasks (whole warps per CV)
    int base[kMaxCv + 1];
    base[0] = 0;
    for (int k = 0; k < d; ++k) base[k + 1] = base[k] + align32((wd.cv[k].type == ABP_CV_COM_DIST ? 2 : 1) * nt);
    const int ntask = base[d];
    const bool overlap = ntask < g.G;
    if (g.t == 0) *badp = 0;
    g.sync();
    // a mask per thread, OR-ed over the warp, one shared-memory OR per warp
    auto finite = [&](int t, int T) {
      unsigned mine = 0;
      Iter2 it(t, T, natoms);
      while (it.j < nt) {
        R4 p[4];
        int jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          jj[u] = it.j;
          if (it.j < nt) {
            p[u] = xs[it.j * xst + it.i];
            it.next();
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (jj[u] < nt && !finite_rec<Real>(p[u])) mine |= 1u << jj[u];
      }
      mine = __reduce_or_sync(0xffffffffu, mine);
      if (g.lane == 0 && mine) atomicOr(badp, mine);
    };
    if (!overlap) {
      finite(g.t, g.G);
      g.sync();
      for (Iter2 it(g.t, g.G, nt); it.j < d; it.next())
        window_cv<Real>(fx, xs + it.i * xst, it.j, (dmask >> it.i) & 1, st[it.i]);
    } else if (g.t < ntask) {
      int k = 0;
      while (k + 1 < d && g.t >= base[k + 1]) ++k;
      const int r = g.t - base[k];
      if (wd.cv[k].type == ABP_CV_COM_DIST) {
        const int j = min(r >> 1, nt - 1);
        window_com2<Real>(fx, xs + j * xst, k, (dmask >> j) & 1, (r >> 1) < nt, r & 1, st[j]);
      } else if (r < nt) {
        window_cv<Real>(fx, xs + r * xst, k, (dmask >> r) & 1, st[r]);
      }
    } else {
      finite(g.t - ntask, g.G - ntask);
    }
    g.sync();
    const unsigned bad = *badp;
    if (g.t == 0 && bad) atomicAdd(&ctr->nonfinite, __popc(bad));
    for (int j = g.t; j < nt; j += g.G)
      if (!((bad >> j) & 1)) step_flags<Real>(d, (dmask >> j) & 1, st[j]);
    g.sync();
  }

  // a2 .. a4 of window w on the grid: deposits in step order, each preceded
  // by a4 of the steps before it; the first deposit's tables and height are
  // formed while the steps before it interpolate (same grid for both)
  template <int UNR, int DIM>
  __device__ __forceinline__ void chain(const Grp &g, int w) const {
    if (fx->wd.method == ABP_METHOD_MABP) {
      if (box && chain_mabp<DIM>(g, w)) return;
    } else if constexpr (DIM < 3) {
      if (box && chain_one<DIM>(g, w)) return;
    }
    chain_seq<UNR, DIM>(g, w);
  }

  // A well-tempered window with exactly one deposit whose stencil box has at
  // most one node per thread: every grid read of the window in one round --
  // each step's 2^d corners into registers, the deposit's box into shared
  // memory by cp.async -- all from the grid before the deposit. The deposit
  // step's corners give the height (a2); the box is updated from shared
  // memory and stored to the grid (a3); steps before the deposit interpolate
  // their corners as read, steps from it on after applying the deposit to
  // the corners inside its box, with the same arithmetic as the stored nodes
  // (the same bits as reading them back). Returns false (nothing done) for
  // any other window. (Larger boxes go through chain_seq: measured faster,
  // the per-thread copies then cost more than the round trips they save.)
  template <int DIM>
  __device__ bool chain_one(const Grp &g, int w) const {
    static_assert(DIM <= 2, "one-round chain: 1D and 2D grids");
    const WalkerDev &wd = fx->wd;
    const GridDev &gd = wd.g;
    constexpr int d = DIM, NC = 1 << DIM;
    constexpr int rb = DIM > 1 ? 32 : 16;  // node record bytes
    const int nt = nt_of(w), t0 = w * W;
    StepRec<Real> *st = steps_of(w);
    const unsigned bad = fx->winbad[w % 3];
    const unsigned gdep = window_dmask(step0, t0, nt, wd.stride) & ~bad;
    if (__popc(gdep) != 1) return false;
    const int first = __ffs(gdep) - 1;
    const int s0 = 2 * wd.R[0] + 1, s1 = d > 1 ? 2 * wd.R[1] + 1 : 1;
    if (s0 * s1 > g.G) return false;
    // first node of the box per axis (unwrapped: the node below u, plus the
    // centre offset, minus R)
    const int b0 = st[first].da[0] + st[first].dc[0] - wd.R[0];
    const int b1 = d > 1 ? st[first].da[1] + st[first].dc[1] - wd.R[1] : 0;
    window_dep_axis<Real>(g, fx, st[first]);
    unsigned char *grid = reinterpret_cast<unsigned char *>(gd.rec);
    // the round: the box (node o0 + s0 o1 at that record of `box`) ...
    for (Iter2 it(g.t, g.G, s0); it.j < s1; it.next()) {
      const long long off = box_node_off<DIM>(gd, b0, b1, it.i, it.j, rb);
      if (off < 0) continue;
      unsigned char *dst = box + (size_t)(it.i + s0 * it.j) * rb;
      cp_async16(dst, grid + off);
      if (rb == 32) cp_async16(dst + 16, grid + off + 16);
    }
    cp_async_commit();
    // ... and the corners of this thread's step
    const int jstep = g.t;
    const bool mine = jstep < nt && !((bad >> jstep) & 1);
    float4 ca[NC], cb[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ca[c] = cb[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mine) interp_load<Real, DIM>(wd, st[jstep], ca, cb);
    g.sync();  // the deposit's axis state
    build_tables<Real>(g, fx);
    if (jstep == first) window_height_regs<Real, DIM>(fx, st[first], ca, cb, step0 + t0 + first, log);
    cp_async_wait_all();
    g.sync();  // tables, height and box
    const Real h = fx->hf;
    for (Iter2 it(g.t, g.G, s0); it.j < s1; it.next()) {
      const int o0 = it.i, o1 = it.j;
      const long long off = box_node_off<DIM>(gd, b0, b1, o0, o1, rb);
      if (off < 0) continue;
      const unsigned sa = (unsigned)__cvta_generic_to_shared(box + (size_t)(o0 + s0 * o1) * rb);
      float4 ra = lds128(sa), rbv = rb == 32 ? lds128(sa + 16) : make_float4(0.f, 0.f, 0.f, 0.f);
      Real G = h * fx->tabG[0][o0];
      if (d > 1) G = G * fx->tabG[1][o1];
      rmw_regs<Real>(d, ra, rbv, G, fx->tabD[0][o0], d > 1 ? fx->tabD[1][o1] : (Real)0, (Real)0);
      float4 *q = reinterpret_cast<float4 *>(grid + off);
      q[0] = ra;
      if (rb == 32) q[1] = rbv;
    }
    if (mine) {
      StepRec<Real> &sj = st[jstep];
      if (jstep >= first) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          int o[2] = {0, 0};
          bool in = true;
#pragma unroll
          for (int k = 0; k < d; ++k) {
            const int n = gd.n[k];
            int r = (((c >> k) & 1) ? sj.i1[k] : sj.i0[k]) - (k ? b1 : b0);
            if (gd.periodic[k]) {
              if (r < 0) r += n;
              if (r >= n) r -= n;
            }
            in = in && r >= 0 && r <= 2 * wd.R[k];
            o[k] = r;
          }
          if (!in) continue;
          Real G = h * fx->tabG[0][o[0]];
          if (d > 1) G = G * fx->tabG[1][o[1]];
          rmw_regs<Real>(d, ca[c], cb[c], G, fx->tabD[0][o[0]], d > 1 ? fx->tabD[1][o[1]] : (Real)0, (Real)0);
        }
      }
      interp_combine<Real, DIM>(wd, sj, ca, cb);
    }
    g.sync();
    if (w + 1 == nwin && g.t == 0) write_state(st, nt, bad);
    return true;
  }

  // mABP: the window's deposits through shared memory. Every hill has the
  // fixed height w and sits on its step's nearest node, so no deposit depends
  // on a look-up: the union of the window's stencil boxes is copied into
  // shared memory, the hills are applied there one after another (the same
  // compensated additions as chain_seq's, so the same bits), each step reads
  // its node there once the hills up to its own are in, and the box is
  // written back. Steps whose node lies outside the union read the grid.
  // Returns false (nothing done) when the union does not fit.
  template <int DIM>
  __device__ bool chain_mabp(const Grp &g, int w) const {
    const WalkerDev &wd = fx->wd;
    const GridDev &gd = wd.g;
    constexpr int d = DIM;
    const int nt = nt_of(w), t0 = w * W, rb = gd.rec_bytes;
    StepRec<Real> *st = steps_of(w);
    const unsigned bad = fx->winbad[w % 3];
    const unsigned gdep = window_dmask(step0, t0, nt, wd.stride) & ~bad;
    const int first = gdep ? __ffs(gdep) - 1 : nt;
    int org[3] = {0, 0, 0}, span[3] = {1, 1, 1};
    long long nodes = gdep ? 1 : 0;
    if (gdep) {
      for (int k = 0; k < d; ++k) {
        const int n = gd.n[k], c0 = st[first].da[k];
        int lo = 0, hi = 0;
        for (unsigned m = gdep; m; m &= m - 1) {
          int dd = st[__ffs(m) - 1].da[k] - c0;
          if (gd.periodic[k]) {
            dd %= n;
            if (dd < 0) dd += n;
            if (2 * dd > n) dd -= n;
          }
          lo = min(lo, dd);
          hi = max(hi, dd);
        }
        lo -= wd.R[k];
        hi += wd.R[k];
        if (gd.periodic[k]) {
          if (hi - lo + 1 >= n) {
            org[k] = 0;
            span[k] = n;
          } else {
            org[k] = ((c0 + lo) % n + n) % n;
            span[k] = hi - lo + 1;
          }
        } else {
          org[k] = max(c0 + lo, 0);
          span[k] = min(c0 + hi, n - 1) - org[k] + 1;
        }
        nodes *= span[k];
      }
      if (nodes * rb > kMabpBoxBytes) return false;
    }
    // box index of a node, or -1 outside the box
    auto box_index = [&](const int *j) -> int {
      int idx = 0, mul = 1;
      for (int k = 0; k < d; ++k) {
        int r = j[k] - org[k];
        if (gd.periodic[k] && r < 0) r += gd.n[k];
        if (r < 0 || r >= span[k]) return -1;
        idx += mul * r;
        mul *= span[k];
      }
      return idx;
    };
    // raw histograms of a step's node, kept in V / dv until the window's end
    auto raw_copy = [&](StepRec<Real> &s, const unsigned char *p) {
      Real v[4] = {0, 0, 0, 0};
      float4 ra, rbv;
      rec_load<DIM>(p, ra, rbv);
      rec_vals<Real, DIM>(ra, rbv, v);
      s.V = v[0];
      for (int k = 0; k < 3; ++k) s.dv[k] = v[1 + k];
    };
    const unsigned char *rec = reinterpret_cast<const unsigned char *>(gd.rec);
    auto node_ptr = [&](int idx) -> const unsigned char * {
      long long node = 0, mul = 1;
      int r = idx;
      for (int k = 0; k < d; ++k) {
        const int q = r % span[k];
        r /= span[k];
        int j = org[k] + q;
        if (j >= gd.n[k]) j -= gd.n[k];
        node += mul * j;
        mul *= gd.n[k];
      }
      return rec + chk_node(gd, node) * rb;
    };
    // steps read from the box (bit j), the rest from the grid
    unsigned inbox = 0;
    if (gdep)
      for (int j = 0; j < nt; ++j)
        if (!((bad >> j) & 1) && box_index(st[j].da) >= 0) inbox |= 1u << j;
    // tables of the node-centred hill (the same for every deposit)
    if (g.t < d) {
      fx->da[g.t] = 0;
      fx->dc[g.t] = 0;
      fx->df[g.t] = 0;
    }
    g.sync();
    build_tables<Real>(g, fx);
    // the box in; steps outside it read the grid
    for (int i = g.t; i < nodes; i += g.G) {
      const float4 *src = reinterpret_cast<const float4 *>(node_ptr(i));
      float4 *dst = reinterpret_cast<float4 *>(box + (size_t)i * rb);
      dst[0] = src[0];
      if (rb == 32) dst[1] = src[1];
    }
    for (int j = g.t; j < nt; j += g.G)
      if (!((bad >> j) & 1) && !((inbox >> j) & 1)) interp_one<Real, DIM>(wd, st[j]);
    g.sync();
    for (int j = g.t; j < first; j += g.G)
      if ((inbox >> j) & 1) raw_copy(st[j], box + (size_t)box_index(st[j].da) * rb);
    const Real h = (Real)wd.w;
    const int s0 = 2 * wd.R[0] + 1, s1 = d > 1 ? 2 * wd.R[1] + 1 : 1, s2 = d > 2 ? 2 * wd.R[2] + 1 : 1;
    const int sp01 = s0 * s1;
    for (unsigned m = gdep; m; m &= m - 1) {
      const int j = __ffs(m) - 1;
      const unsigned rest = m & (m - 1);
      const int next = rest ? __ffs(rest) - 1 : nt;
      g.sync();  // the hills and look-ups before this hill are done
      // box-relative position of the hill's first node, per axis
      // (on a periodic axis taken into [0, n), so that one wrap suffices below)
      int base[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) {
        base[k] = st[j].da[k] - wd.R[k] - org[k];
        if (gd.periodic[k]) base[k] = ((base[k] % gd.n[k]) + gd.n[k]) % gd.n[k];
      }
      const bool centre_in = (inbox >> j) & 1;
      // stencil positions (o0 fastest), advanced without division
      Iter2 it(g.t, g.G, s0);
      for (int idx = g.t; idx < sp01 * s2; idx += g.G, it.next()) {
        const int o0 = it.i, o12 = it.j, o1 = d > 2 ? o12 % s1 : o12, o2 = d > 2 ? o12 / s1 : 0;
        const int o[3] = {o0, o1, o2};
        int bi = 0, mul = 1;
        bool in = true;
        for (int k = 0; k < d; ++k) {
          const int n = gd.n[k];
          int r = base[k] + o[k];  // node - org
          if (gd.periodic[k]) {
            if (r >= n) r -= n;
          } else {
            const int jn = r + org[k];
            in = in && jn >= 0 && jn < n;
          }
          in = in && r >= 0 && r < span[k];
          bi += mul * r;
          mul *= span[k];
        }
        if (!in) continue;
        Real G = h * fx->tabG[0][o0];
        if (d > 1) G = G * fx->tabG[1][o1];
        if (d > 2) G = G * fx->tabG[2][o2];
        const Real d0 = fx->tabD[0][o0], d1 = d > 1 ? fx->tabD[1][o1] : (Real)0,
                   d2 = d > 2 ? fx->tabD[2][o2] : (Real)0;
        unsigned char *p = box + (size_t)bi * rb;
        // the record through shared-memory loads and stores
        const unsigned sa = (unsigned)__cvta_generic_to_shared(p);
        float4 ra = lds128(sa), rbv = rb == 32 ? lds128(sa + 16) : make_float4(0, 0, 0, 0);
        rmw_regs<Real>(d, ra, rbv, G, d0, d1, d2);
        sts128(sa, ra);
        if (rb == 32) sts128(sa + 16, rbv);
        // the hill's own step reads its centre right after it
        if (centre_in && o0 == wd.R[0] && (d < 2 || o1 == wd.R[1]) && (d < 3 || o2 == wd.R[2])) raw_copy(st[j], p);
      }
      if (g.t == g.G - 1 && log.rec) window_height<Real, DIM>(fx, st[j], step0 + t0 + j, log);
      if (next > j + 1) {  // steps between this hill and the next read after it
        g.sync();
        for (int q = j + 1 + g.t; q < next; q += g.G)
          if ((inbox >> q) & 1) raw_copy(st[q], box + (size_t)box_index(st[q].da) * rb);
      }
    }
    g.sync();
    // the box out; the raw histograms of the steps read in it become the bias
    for (int i = g.t; i < nodes; i += g.G) {
      float4 *dst = reinterpret_cast<float4 *>(const_cast<unsigned char *>(node_ptr(i)));
      const float4 *src = reinterpret_cast<const float4 *>(box + (size_t)i * rb);
      dst[0] = src[0];
      if (rb == 32) dst[1] = src[1];
    }
    for (int j = g.t; j < nt; j += g.G)
      if ((inbox >> j) & 1) {
        Real acc[4] = {st[j].V, st[j].dv[0], st[j].dv[1], st[j].dv[2]};
        finish_lookup<Real>(wd, st[j], acc);
      }
    g.sync();
    if (w + 1 == nwin && g.t == 0) write_state(st, nt, bad);
    return true;
  }

  // the walker's state after the call's last step
  __device__ __forceinline__ void write_state(const StepRec<Real> *st, int nt, unsigned bad) const {
    const WalkerDev &wd = fx->wd;
    const StepRec<Real> &s = st[nt - 1];
    if ((bad >> (nt - 1)) & 1) {
      wd.state->flags = ABP_WFLAG_NONFINITE;
    } else {
      WalkerState ws;
      for (int k = 0; k < 3; ++k) {
        ws.s[k] = k < wd.g.d ? (double)s.s[k] + (double)s.sl[k] : 0.0;
        ws.dV[k] = k < wd.g.d ? (double)s.dv[k] : 0.0;
      }
      ws.V = (double)s.V;
      ws.flags = s.flags;
      ws.pad = 0;
      ws.step = step0 + last;
      *wd.state = ws;
    }
  }

  template <int UNR, int DIM>
  __device__ __forceinline__ void chain_seq(const Grp &g, int w) const {
    const WalkerDev &wd = fx->wd;
    const int nt = nt_of(w), t0 = w * W;
    StepRec<Real> *st = steps_of(w);
    const unsigned bad = fx->winbad[w % 3];
    const unsigned gdep = window_dmask(step0, t0, nt, wd.stride) & ~bad;  // non-finite steps deposit nothing
    const int first = gdep ? __ffs(gdep) - 1 : nt;
    if (gdep) {
      window_dep_axis<Real>(g, fx, st[first]);
      g.sync();
    }
    for (int j = g.t; j < first; j += g.G)
      if (!((bad >> j) & 1)) interp_one<Real, DIM>(wd, st[j]);
    if (gdep) {
      build_tables<Real>(g, fx);
      if (g.t == g.G - 1) window_height<Real, DIM>(fx, st[first], step0 + t0 + first, log);
    }
    g.sync();
    int seg = first;
    for (unsigned m = gdep; m; m &= m - 1) {
      const int j = __ffs(m) - 1;
      if (j != first) {
        for (int q = seg + g.t; q < j; q += g.G)
          if (!((bad >> q) & 1)) interp_one<Real, DIM>(wd, st[q]);
        window_dep_axis<Real>(g, fx, st[j]);
        g.sync();
        build_tables<Real>(g, fx);
        if (g.t == g.G - 1) window_height<Real, DIM>(fx, st[j], step0 + t0 + j, log);
        g.sync();
      }
      deposit_stencil<Real, false, UNR>(g, fx, L, nullptr);
      g.sync();
      seg = j;
    }
    for (int q = seg + g.t; q < nt; q += g.G)
      if (!((bad >> q) & 1)) interp_one<Real, DIM>(wd, st[q]);
    g.sync();
    if (w + 1 == nwin && g.t == 0) write_state(st, nt, bad);
  }

  // C: a5 per (step, atom), stored as it is formed
  __device__ __forceinline__ void forces(const Grp &g, int w) const {
    const int nt = nt_of(w), t0 = w * W, natoms = fx->wd.natoms;
    const StepRec<Real> *st = steps_of(w);
    const unsigned bad = fx->winbad[w % 3];
    R4 *fout = out ? reinterpret_cast<R4 *>(out) : reinterpret_cast<R4 *>(fx->wd.fbuf);
    // FP32 walkers: one atom per thread (its terms in registers) over every
    // nl-th step; FP64 walkers, whose C runs on the chain half, measured
    // faster with one (step, atom) pair per thread
    if (sizeof(Real) == 4 && !serial_out && natoms <= g.G) {
      const int nl = g.G / natoms, a = g.t % natoms, lane0 = g.t / natoms;
      if (lane0 < nl) {
        const AtomTerm<Real> *ta = terms + a * kAtomTerms;
        const int ne = cnt[a];
        Real tw[kAtomTerms];
        int toff[kAtomTerms];
#pragma unroll
        for (int q = 0; q < kAtomTerms; ++q) {
          tw[q] = q < ne ? ta[q].w : (Real)0;
          toff[q] = q < ne ? ta[q].off : 0;
        }
        for (int j = lane0; j < nt; j += nl) {
          const long long t = (long long)t0 + j;
          if (!out && t != last) continue;  // the walker's own buffer keeps the last step
          R4 *fo = fout + foff + (out ? t * fstride : 0) + a;
          if ((bad >> j) & 1) {
            if (mode == ABP_FORCES_OVERWRITE) *fo = make_rec<Real>(0, 0, 0, 0);
            continue;
          }
          // the atom's terms in order, as atom_force sums them
          const Real *J = &st[j].jac[0][0];
          Real f0 = 0, f1 = 0, f2 = 0;
#pragma unroll
          for (int q = 0; q < kAtomTerms; ++q)
            if (q < ne) {
              const Real *v = J + toff[q];
              f0 += tw[q] * v[0];
              f1 += tw[q] * v[1];
              f2 += tw[q] * v[2];
            }
          store_force_stream<Real>(fo, make_rec<Real>(f0, f1, f2, 0), mode);
        }
      }
    } else if (!serial_out) {
      for (Iter2 it(g.t, g.G, natoms); it.j < nt; it.next()) {
        const long long t = (long long)t0 + it.j;
        if (!out && t != last) continue;  // the walker's own buffer keeps the last step
        R4 *fo = fout + foff + (out ? t * fstride : 0) + it.i;
        if ((bad >> it.j) & 1) {
          if (mode == ABP_FORCES_OVERWRITE) *fo = make_rec<Real>(0, 0, 0, 0);
        } else {
          store_force_stream<Real>(fo, atom_force<Real>(cnt, terms, it.i, st[it.j]), mode);
        }
      }
    } else {
      // forces of several steps to one address: added in step order
      for (int i = g.t; i < natoms; i += g.G)
        for (int j = 0; j < nt; ++j) {
          R4 *fo = fout + foff + i;
          if ((bad >> j) & 1) {
            if (mode == ABP_FORCES_OVERWRITE) *fo = make_rec<Real>(0, 0, 0, 0);
          } else {
            store_force<Real>(fo, atom_force<Real>(cnt, terms, i, st[j]), mode);
          }
        }
    }
  }
};

// The windowed form's driver. Iteration w runs A of window w + 1 and C of
// window w - 1 (grid-independent) beside the grid chain of window w; the
// three touch different StepRec arrays. A group of two or more warps splits
// in halves on their own named barriers, the first half taking A and C (and
// the coordinate copies), the second the chain; a one-warp group runs the
// three in turn.
template <typename Real, int UNR, int DIM>
__device__ __forceinline__ void walker_window(const Grp &g, GroupFixed<Real> *fx, unsigned char *dyn,
                                              const GroupLayout &L, const RunArgs &a, int widx) {
  using R4 = typename Rec4<Real>::T;
  WindowCtx<Real> c;
  c.fx = fx;
  c.L = L;
  c.coords = a.coords;
  c.out = a.forces;
  c.cstride = a.cstride;
  c.fstride = a.fstride;
  c.nsteps = a.nsteps;
  c.xst = L.xstride;
  c.ctr = a.ctr;
  c.log = a.log;
  c.xb[0] = reinterpret_cast<R4 *>(dyn + L.xs0);
  c.xb[1] = reinterpret_cast<R4 *>(dyn + L.xs1);
  c.steps = reinterpret_cast<StepRec<Real> *>(dyn + L.steps);
  c.cnt = reinterpret_cast<int *>(dyn + L.atoms);
  c.terms = reinterpret_cast<AtomTerm<Real> *>(dyn + L.atoms + align16(fx->wd.natoms * 4));
  c.coff = a.coff[widx];
  c.foff = a.forces ? a.foff[widx] : 0;
  c.step0 = a.wstep ? a.wstep[widx] : a.step0;
  c.last = (long long)a.nsteps - 1;
  c.W = L.win;
  c.nwin = (a.nsteps + L.win - 1) / L.win;
  c.mode = a.forces ? a.mode : ABP_FORCES_OVERWRITE;
  c.serial_out = a.forces && a.fstride == 0;
  c.stream = l2_evict_first();
  c.box = L.box ? dyn + L.tile : nullptr;
  // the two halves (or the whole warp twice)
  const bool split = g.G >= 64;
  Grp gx = g, gy = g;
  if (split) {
    gx.G = gy.G = g.G / 2;
    gx.nwarps = gy.nwarps = g.nwarps / 2;
    gx.gid = a.groups_per_cta + 2 * g.gid;  // named barriers after the groups' own (gid + 1)
    gy.gid = gx.gid + 1;
    gy.t = g.t - gx.G;
    gy.warp = g.warp - gx.nwarps;
  }
  const bool isx = !split || g.t < g.G / 2, isy = !split || !isx;
  build_atom_terms<Real>(g, fx, c.cnt, c.terms);
  // Each phase has one call site, so that one copy of its code computes
  // every window's steps (the same bits whichever window a step falls in).
  if (split && a.groups_per_cta == 1) {
    // The halves decoupled: A hands window i to the chain through barrier
    // FULL[i % 3] (A arrives, the chain waits), the chain hands it back for
    // C through DONE[i % 3]; A runs up to two windows ahead of C, so a
    // window whose chain is long (a deposit) and one whose A is long even
    // out. (The three StepRec slots are free again by the time A reuses
    // them: A has waited on DONE for window i - 3 and run its C.)
    // FP64 walkers: A's FP64 arithmetic is the long half, so the chain half
    // runs C (measured on the one-walker FP64 workload; FP32 the other way)
    constexpr bool kCForChain = sizeof(Real) == 8;
    const int full0 = 3 * a.groups_per_cta + 1, done0 = full0 + 3;
    if (isx) {
      c.prefetch(gx, 0);
      if (c.nwin > 1) c.prefetch(gx, 1);
      for (int i = 0; i < c.nwin + 2; ++i) {
        if (i < c.nwin) {
          // window i's coordinates (window i + 1's may still be in flight)
          if (i + 1 < c.nwin)
            asm volatile("cp.async.wait_group 1;" ::: "memory");
          else
            cp_async_wait_all();
          gx.sync();
          c.cvs(gx, i);
          if (i + 2 < c.nwin) c.prefetch(gx, i + 2);  // into window i's buffer, read by now
          bar_arrive(full0 + i % 3, g.G);
        }
        if (i >= 2) {
          bar_wait(done0 + (i - 2) % 3, g.G);
          if (!kCForChain) c.forces(gx, i - 2);
        }
      }
    } else {
      for (int w = 0; w < c.nwin; ++w) {
        bar_wait(full0 + w % 3, g.G);
        c.template chain<UNR, DIM>(gy, w);
        if (kCForChain) c.forces(gy, w);
        bar_arrive(done0 + w % 3, g.G);
      }
    }
    return;
  }
  // Lockstep: iteration w runs A of window w + 1 and C of window w - 1
  // beside the chain of window w; iteration -1 only evaluates window 0's CVs.
  if (isx) c.prefetch(gx, 0);
  for (int w = -1; w <= c.nwin; ++w) {
    if (isx) {
      if (w + 1 < c.nwin) {
        cp_async_wait_all();  // window w + 1's coordinates
        gx.sync();
        if (w + 2 < c.nwin) c.prefetch(gx, w + 2);  // into the buffer window w used
        c.cvs(gx, w + 1);
      }
      if (w >= 1) c.forces(gx, w - 1);
    }
    if (isy && w >= 0 && w < c.nwin) c.template chain<UNR, DIM>(gy, w);
    g.sync();
  }
}

template <typename Real, bool TILE>
__device__ __forceinline__ void run_body(const RunArgs &a) {
  extern __shared__ __align__(32) unsigned char smem[];
  const int gid = threadIdx.x / a.G;
  const int slot = blockIdx.x * a.groups_per_cta + gid;
  if (slot >= a.nw) return;
  Grp g;
  g.G = a.G;
  g.gid = gid;
  g.t = threadIdx.x - gid * a.G;
  g.lane = threadIdx.x & 31;
  g.warp = g.t >> 5;
  g.nwarps = a.G >> 5;
  unsigned char *base = smem + (size_t)gid * a.group_bytes;
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(base);
  unsigned char *dyn = base + fixed_bytes<Real>();
  const TableEntry te = a.table[slot];
  copy_desc<Real>(g, &fx->wd, te.wd);
  g.sync();
  const GroupLayout L = layout_of<Real>(fx, g.nwarps, TILE ? a.tile_budget : 0, false);
  setup_lists<Real>(g, fx, dyn + L.lists);
  g.sync();
  if (TILE && L.tile_nodes > 0)
    walker_steps<Real, true>(g, fx, dyn, L, a, te.idx);
  else
    walker_steps<Real, false>(g, fx, dyn, L, a, te.idx);
}

template <typename Real, bool TILE>
__global__ void __launch_bounds__(256, 1) k_run(RunArgs a) {
  run_body<Real, TILE>(a);
}

// The same kernel compiled for two resident 256-thread CTAs per SM (at most
// 128 registers per thread): more warps to hide latency for batches whose
// walkers are busy in long CN pair loops. Chosen by ABP_TUNE_LEAN.
__global__ void __launch_bounds__(256, 2) k_run_lean(RunArgs a) { run_body<float, false>(a); }

// The windowed form (walkers whose CVs are COM distances, dihedrals or small
// RMSDs), in kernels of its own, one per grid dimension DIM: each keeps only
// its own code in the instruction cache.
template <typename Real, int UNR, int DIM>
__global__ void __launch_bounds__(256, 1) k_win(RunArgs a) {
  extern __shared__ __align__(32) unsigned char smem[];
  const int gid = threadIdx.x / a.G;
  const int slot = blockIdx.x * a.groups_per_cta + gid;
  if (slot >= a.nw) return;
  Grp g;
  g.G = a.G;
  g.gid = gid;
  g.t = threadIdx.x - gid * a.G;
  g.lane = threadIdx.x & 31;
  g.warp = g.t >> 5;
  g.nwarps = a.G >> 5;
  unsigned char *base = smem + (size_t)gid * a.group_bytes;
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(base);
  unsigned char *dyn = base + fixed_bytes<Real>();
  const TableEntry te = a.table[slot];
  copy_desc<Real>(g, &fx->wd, te.wd);
  g.sync();
  const GroupLayout L = layout_of<Real>(fx, g.nwarps, 0, true);
  if (L.win == 0 || fx->wd.g.d != DIM) return;  // the host sends only eligible walkers of DIM CVs here
  setup_lists<Real>(g, fx, dyn + L.lists);
  g.sync();
  walker_window<Real, UNR, DIM>(g, fx, dyn, L, a, te.idx);
}

cudaError_t launch_run(const RunArgs &a, int fp64, cudaStream_t st) {
  const int threads = a.G * a.groups_per_cta;
  const int blocks = (a.nw + a.groups_per_cta - 1) / a.groups_per_cta;
  const size_t smem = (size_t)a.group_bytes * a.groups_per_cta;
  if (a.nw == 0) return cudaSuccess;
  cudaError_t e;
  if (a.window) {
    void (*k)(RunArgs);
    if (fp64)
      k = a.window == 1 ? k_win<double, 4, 1> : a.window == 2 ? k_win<double, 4, 2> : k_win<double, 4, 3>;
    else
      k = a.window == 1 ? k_win<float, 7, 1> : a.window == 2 ? k_win<float, 7, 2> : k_win<float, 7, 3>;
    e = smem_attr(reinterpret_cast<const void *>(k), smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
  }
  if (fp64) {
    e = smem_attr(reinterpret_cast<const void *>(k_run<double, false>), smem);
    if (e != cudaSuccess) return e;
    k_run<double, false><<<blocks, threads, smem, st>>>(a);
  } else if (a.lean && a.tile_budget == 0) {
    e = smem_attr(reinterpret_cast<const void *>(k_run_lean), smem);
    if (e != cudaSuccess) return e;
    k_run_lean<<<blocks, threads, smem, st>>>(a);
  } else if (a.tile_budget > 0) {
    e = smem_attr(reinterpret_cast<const void *>(k_run<float, true>), smem);
    if (e != cudaSuccess) return e;
    k_run<float, true><<<blocks, threads, smem, st>>>(a);
  } else {
    e = smem_attr(reinterpret_cast<const void *>(k_run<float, false>), smem);
    if (e != cudaSuccess) return e;
    k_run<float, false><<<blocks, threads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

bool window_eligible(const WalkerDev &hd, int fp64) {
  return window_steps(hd.natoms, hd.cv, hd.g.d, fp64 ? 32 : 16) > 0;
}

int run_group_bytes(const WalkerDev &hd, int fp64, int G, int tile_budget, bool window) {
  GroupLayout L = group_layout(hd.natoms, hd.cv, hd.g, hd.R, G / 32, fp64 ? 32 : 16, tile_budget, window,
                               hd.method == ABP_METHOD_MABP);
  return align32(group_fixed_bytes(fp64) + L.total);
}

// ---------------------------------------------------------------- plain form
//
// Scratch kept in the walker's global jscratch buffer between launches:
// PlainScratch, then for each COORD CV its dCN/dx records (A list, B list).

template <typename Real>
struct PlainScratch {
  Real sh[kMaxCv], sl[kMaxCv];
  Real com_u[kMaxCv][3];
  Real dih_g[kMaxCv][4][3];
  int flags;
  int bad;
};

template <typename Real>
__host__ __device__ constexpr int plain_head_bytes() {
  return (int)((sizeof(PlainScratch<Real>) + 31) & ~(size_t)31);
}

int plain_scratch_bytes(int fp64, const CvDev *cv, int ncv) {
  int rsz = fp64 ? 32 : 16;
  int b = fp64 ? plain_head_bytes<double>() : plain_head_bytes<float>();
  for (int k = 0; k < ncv; ++k)
    if (cv[k].type == ABP_CV_COORD) b += (cv[k].na + cv[k].nb) * rsz;
  return b;
}

template <typename Real>
__device__ __forceinline__ Grp cta_group() {
  Grp g;
  g.G = blockDim.x;
  g.gid = 0;
  g.t = threadIdx.x;
  g.lane = threadIdx.x & 31;
  g.warp = threadIdx.x >> 5;
  g.nwarps = blockDim.x >> 5;
  return g;
}

template <typename Real>
__device__ GroupLayout plain_prologue(const Grp &g, GroupFixed<Real> *fx, const WalkerDev *wdp, unsigned char *dyn) {
  copy_desc<Real>(g, &fx->wd, wdp);
  g.sync();
  GroupLayout L = layout_of<Real>(fx, g.nwarps, 0, false);
  setup_lists<Real>(g, fx, dyn + L.lists);
  if (g.t == 0) {
    fx->flags = 0;
    fx->clamped = 0;
  }
  g.sync();
  return L;
}

// a1 for one walker; results to the walker's scratch.
template <typename Real>
__global__ void __launch_bounds__(256) k_plain_cv(const WalkerDev *wdp, const void *coords, const long long *coff,
                                                  int widx) {
  using R4 = typename Rec4<Real>::T;
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = cta_group<Real>();
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(smem);
  unsigned char *dyn = smem + fixed_bytes<Real>();
  const GroupLayout L = plain_prologue<Real>(g, fx, wdp, dyn);
  const WalkerDev &wd = fx->wd;
  R4 *xs = reinterpret_cast<R4 *>(dyn + L.xs0);
  unsigned char *cnmem = dyn + L.cn;
  const R4 *xin = reinterpret_cast<const R4 *>(coords) + coff[widx];
  int bad = 0;
  for (int i = g.t; i < wd.natoms; i += g.G) {
    R4 p = xin[i];
    xs[i] = p;
    bad |= finite_rec<Real>(p) ? 0 : 1;
  }
  PlainScratch<Real> *ps = reinterpret_cast<PlainScratch<Real> *>(wd.jscratch);
  if (grp_any<Real>(g, fx, bad)) {
    if (g.t == 0) {
      ps->bad = 1;
      ps->flags = ABP_WFLAG_NONFINITE;
    }
    return;
  }
  g.sync();
  eval_cvs<Real>(g, fx, xs, cnmem);
  if (g.t == 0) {
    ps->bad = 0;
    ps->flags = fx->flags;
    for (int k = 0; k < kMaxCv; ++k) {
      ps->sh[k] = fx->sh[k];
      ps->sl[k] = fx->sl[k];
      for (int q = 0; q < 3; ++q) ps->com_u[k][q] = fx->com_u[k][q];
      for (int b = 0; b < 4; ++b)
        for (int q = 0; q < 3; ++q) ps->dih_g[k][b][q] = fx->dih_g[k][b][q];
    }
  }
  R4 *jout = reinterpret_cast<R4 *>(reinterpret_cast<unsigned char *>(wd.jscratch) + plain_head_bytes<Real>());
  for (int k = 0; k < wd.g.d; ++k) {
    const CvDev &c = wd.cv[k];
    if (c.type != ABP_CV_COORD) continue;
    const R4 *jl = reinterpret_cast<const R4 *>(cn_slot<Real>(cnmem, wd, k, g.nwarps));
    for (int i = g.t; i < c.na + c.nb; i += g.G) jout[i] = jl[i];
    jout += c.na + c.nb;
  }
}

// a2 + a3 for one walker (launched on deposit steps only).
template <typename Real>
__global__ void __launch_bounds__(256) k_plain_deposit(const WalkerDev *wdp, long long step, DepositLog log) {
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = cta_group<Real>();
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(smem);
  unsigned char *dyn = smem + fixed_bytes<Real>();
  const GroupLayout L = plain_prologue<Real>(g, fx, wdp, dyn);
  const PlainScratch<Real> *ps = reinterpret_cast<const PlainScratch<Real> *>(fx->wd.jscratch);
  if (ps->bad) return;
  if (g.t < kMaxCv) {
    fx->sh[g.t] = ps->sh[g.t];
    fx->sl[g.t] = ps->sl[g.t];
  }
  g.sync();
  if (g.t < fx->wd.g.d) axis_setup<Real>(fx, g.t, true);
  g.sync();
  deposit_step<Real, false>(g, fx, L, nullptr, step, log);
}

// a4 + a5 for one walker.
template <typename Real>
__global__ void __launch_bounds__(256) k_plain_force(const WalkerDev *wdp, void *forces, const long long *foff, int widx,
                                                     int mode, long long step, DevCounters *ctr) {
  using R4 = typename Rec4<Real>::T;
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = cta_group<Real>();
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(smem);
  unsigned char *dyn = smem + fixed_bytes<Real>();
  const GroupLayout L = plain_prologue<Real>(g, fx, wdp, dyn);
  const WalkerDev &wd = fx->wd;
  R4 *fs = reinterpret_cast<R4 *>(dyn + L.fs);
  unsigned char *cnmem = dyn + L.cn;
  const PlainScratch<Real> *ps = reinterpret_cast<const PlainScratch<Real> *>(wd.jscratch);
  R4 *fo = reinterpret_cast<R4 *>(forces) + foff[widx];
  if (ps->bad) {
    if (mode == ABP_FORCES_OVERWRITE)
      for (int i = g.t; i < wd.natoms; i += g.G) fo[i] = make_rec<Real>(0, 0, 0, 0);
    if (g.t == 0) {
      wd.state->flags = ABP_WFLAG_NONFINITE;
      atomicAdd(&ctr->nonfinite, 1);
    }
    return;
  }
  if (g.t == 0) {
    fx->flags = ps->flags | ((step % wd.stride) == 0 ? ABP_WFLAG_DEPOSIT : 0);
    for (int k = 0; k < kMaxCv; ++k) {
      fx->sh[k] = ps->sh[k];
      fx->sl[k] = ps->sl[k];
      for (int q = 0; q < 3; ++q) fx->com_u[k][q] = ps->com_u[k][q];
      for (int b = 0; b < 4; ++b)
        for (int q = 0; q < 3; ++q) fx->dih_g[k][b][q] = ps->dih_g[k][b][q];
    }
  }
  const R4 *jin =
      reinterpret_cast<const R4 *>(reinterpret_cast<const unsigned char *>(wd.jscratch) + plain_head_bytes<Real>());
  for (int k = 0; k < wd.g.d; ++k) {
    const CvDev &c = wd.cv[k];
    if (c.type != ABP_CV_COORD) continue;
    R4 *jl = reinterpret_cast<R4 *>(cn_slot<Real>(cnmem, wd, k, g.nwarps));
    for (int i = g.t; i < c.na + c.nb; i += g.G) jl[i] = jin[i];
    jin += c.na + c.nb;
  }
  for (int i = g.t; i < wd.natoms; i += g.G) fs[i] = make_rec<Real>(0, 0, 0, 0);
  g.sync();
  if (g.t < wd.g.d) axis_setup<Real>(fx, g.t, false);
  g.sync();
  interp_step<Real, false>(g, fx, L, nullptr);
  scatter_forces<Real>(g, fx, fs, cnmem);
  for (int i = g.t; i < wd.natoms; i += g.G) store_force<Real>(fo + i, fs[i], mode);
  if (g.t == 0) write_state<Real>(fx, step);
}

template <typename Real>
static cudaError_t plain_one(const PlainArgs &a, int w, cudaStream_t st) {
  const WalkerDev *wd = a.wd_dev[w];
  const int T = a.threads;
  size_t smem = (size_t)fixed_bytes<Real>() + a.dyn_bytes[w];
  cudaError_t e;
  e = smem_attr(reinterpret_cast<const void *>(k_plain_cv<Real>), smem);
  if (e != cudaSuccess) return e;
  k_plain_cv<Real><<<1, T, smem, st>>>(wd, a.coords, a.coff, w);
  if (a.deposit[w]) {
    e = smem_attr(reinterpret_cast<const void *>(k_plain_deposit<Real>), smem);
    if (e != cudaSuccess) return e;
    k_plain_deposit<Real><<<1, T, smem, st>>>(wd, a.step, a.log);
  }
  e = smem_attr(reinterpret_cast<const void *>(k_plain_force<Real>), smem);
  if (e != cudaSuccess) return e;
  k_plain_force<Real><<<1, T, smem, st>>>(wd, a.forces, a.foff, w, a.mode, a.step, a.ctr);
  return cudaGetLastError();
}

cudaError_t launch_plain(const PlainArgs &a, int fp64, cudaStream_t st) {
  for (int w = 0; w < a.nw; ++w) {
    cudaError_t e = fp64 ? plain_one<double>(a, w, st) : plain_one<float>(a, w, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- abp_forces

template <typename Real>
__global__ void __launch_bounds__(256) k_deliver(const TableEntry *table, int nw, void *forces, const long long *foff,
                                                 int mode) {
  using R4 = typename Rec4<Real>::T;
  const TableEntry te = table[blockIdx.x];
  const WalkerDev *wd = te.wd;
  const int natoms = wd->natoms;
  const R4 *src = reinterpret_cast<const R4 *>(wd->fbuf);
  R4 *dst = reinterpret_cast<R4 *>(forces) + foff[te.idx];
  for (int i = threadIdx.x; i < natoms; i += blockDim.x) store_force<Real>(dst + i, src[i], mode);
}

cudaError_t launch_deliver(const TableEntry *table, int nw, void *forces, const long long *foff, int mode, int fp64,
                           cudaStream_t st) {
  if (nw == 0) return cudaSuccess;
  if (fp64)
    k_deliver<double><<<nw, 128, 0, st>>>(table, nw, forces, foff, mode);
  else
    k_deliver<float><<<nw, 128, 0, st>>>(table, nw, forces, foff, mode);
  return cudaGetLastError();
}

}  // namespace abp
