// abp_kernels.cu -- the kernels of the force call and their launchers:
//   k_run      fused batched form: one walker group per walker, every step
//              a1..a5 for nsteps consecutive MD steps in one launch;
//   k_plain_*  plain form: CV, deposit and interpolation/force as separate
//              single-walker launches (the comparison point);
//   k_deliver  copies each walker's force buffer to the caller (abp_forces).
#include <cuda_runtime.h>

#include "abp_device.cuh"
#include "abp_launch.h"

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
__device__ __forceinline__ unsigned char *cn_slot(unsigned char *cnmem, const WalkerDev &wd, int k, int nwarps) {
  int rsz = (int)sizeof(typename Rec4<Real>::T);
  unsigned char *cur = cnmem;
  for (int q = 0; q < k; ++q) {
    const CvDev &c = wd.cv[q];
    if (c.type == ABP_CV_COORD) cur += (c.na + c.nb) * rsz + ((nwarps * c.na * 3 * (int)sizeof(Real) + 31) & ~31);
  }
  return cur;
}

// a1 for every CV of the walker (coordinates already in xs).
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
      cv_coord<Real>(g, fx, k, xs, jA, jB, lig);
    }
    g.sync();
  }
}

// a2 + a3: height from the grid before the deposit, then the stencil.
template <typename Real>
__device__ void deposit_step(const Grp &g, GroupFixed<Real> *fx, long long step, const DepositLog &log) {
  const WalkerDev &wd = fx->wd;
  build_tables<Real>(g, fx);
  if (g.warp == 0) {
    double out[4];
    interp_corners<double>(wd.g, fx->s, g.lane, out);
    if (g.lane == 0) {
      double h = wd.w * exp(-out[0] * wd.inv_dT);
      fx->hf = (Real)h;
      if (log.rec) {
        unsigned long long slot = atomicAdd(log.count, 1ull);
        if (slot < log.cap) {
          abp_deposit_rec r;
          r.step = step;
          r.walker_id = wd.id;
          for (int k = 0; k < 3; ++k) {
            r.ic[k] = k < wd.g.d ? fx->ic_log[k] : 0;
            r.s[k] = k < wd.g.d ? fx->s[k] : 0.0;
          }
          r.height = h;
          log.rec[slot] = r;
        }
      }
    }
  }
  g.sync();
  deposit_stencil<Real>(g, fx);
  g.sync();
}

// a4: V and dV/ds at s after the deposit (warp 0), broadcast via fx.
template <typename Real>
__device__ void interp_step(const Grp &g, GroupFixed<Real> *fx) {
  const WalkerDev &wd = fx->wd;
  if (g.warp == 0) {
    Real out[4];
    int fl = interp_corners<Real>(wd.g, fx->s, g.lane, out);
    if (g.lane == 0) {
      fx->V = (double)out[0];
      for (int k = 0; k < wd.g.d; ++k) {
        fx->dvds[k] = out[1 + k];
        fx->dV[k] = (double)out[1 + k];
      }
      fx->flags |= fl;
    }
  }
  g.sync();
}

template <typename Real>
__device__ void write_state(const Grp &g, GroupFixed<Real> *fx, long long step) {
  if (g.t != 0) return;
  const WalkerDev &wd = fx->wd;
  WalkerState st;
  for (int k = 0; k < 3; ++k) {
    st.s[k] = k < wd.g.d ? fx->s[k] : 0.0;
    st.dV[k] = k < wd.g.d ? fx->dV[k] : 0.0;
  }
  st.V = fx->V;
  st.flags = fx->flags;
  st.pad = 0;
  st.step = step;
  *wd.state = st;
}

template <typename Real>
__device__ __forceinline__ bool finite_rec(const typename Rec4<Real>::T &p) {
  return isfinite(p.x) && isfinite(p.y) && isfinite(p.z);
}

// nsteps MD steps of one walker (steps a1..a5 each), by one group.
template <typename Real>
__device__ void walker_steps(const Grp &g, GroupFixed<Real> *fx, unsigned char *dyn, const RunArgs &a, int widx) {
  using R4 = typename Rec4<Real>::T;
  const WalkerDev &wd = fx->wd;
  const int natoms = wd.natoms;
  R4 *xs = reinterpret_cast<R4 *>(dyn);
  R4 *fs = xs + natoms;
  unsigned char *cnmem = reinterpret_cast<unsigned char *>(fs + natoms);
  const R4 *cin = reinterpret_cast<const R4 *>(a.coords);
  R4 *fout = a.forces ? reinterpret_cast<R4 *>(a.forces) : reinterpret_cast<R4 *>(wd.fbuf);
  const long long coff = a.coff[widx];
  const long long foff = a.forces ? a.foff[widx] : 0;
  const int mode = a.forces ? a.mode : ABP_FORCES_OVERWRITE;
  for (int t = 0; t < a.nsteps; ++t) {
    const long long step = a.step0 + t;
    const R4 *xin = cin + coff + (long long)t * a.cstride;
    R4 *fo = fout + foff + (a.forces ? (long long)t * a.fstride : 0);
    int bad = 0;
    for (int i = g.t; i < natoms; i += g.G) {
      R4 p = xin[i];
      xs[i] = p;
      fs[i] = make_rec<Real>(0, 0, 0, 0);
      bad |= finite_rec<Real>(p) ? 0 : 1;
    }
    if (g.t == 0) fx->flags = 0;
    Real bv[1] = {(Real)bad};
    grp_sum<1>(g, bv, fx->red);
    g.sync();
    if (bv[0] != 0) {
      // non-finite coordinates: no deposit, zero bias force, state kept
      if (mode == ABP_FORCES_OVERWRITE)
        for (int i = g.t; i < natoms; i += g.G) fo[i] = make_rec<Real>(0, 0, 0, 0);
      if (g.t == 0) {
        wd.state->flags = ABP_WFLAG_NONFINITE;
        atomicAdd(&a.ctr->nonfinite, 1);
      }
      g.sync();
      continue;
    }
    eval_cvs<Real>(g, fx, xs, cnmem);
    const bool dep = (step % wd.stride) == 0;
    if (dep) {
      deposit_step<Real>(g, fx, step, a.log);
      if (g.t == 0) fx->flags |= ABP_WFLAG_DEPOSIT;
    }
    interp_step<Real>(g, fx);
    scatter_forces<Real>(g, fx, fs, cnmem);
    for (int i = g.t; i < natoms; i += g.G) {
      R4 f = fs[i];
      if (mode == ABP_FORCES_ACCUMULATE) {
        R4 o = fo[i];
        o.x += f.x;
        o.y += f.y;
        o.z += f.z;
        fo[i] = o;
      } else {
        fo[i] = make_rec<Real>(f.x, f.y, f.z, 0);
      }
    }
    write_state<Real>(g, fx, step);
    g.sync();
  }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_run(RunArgs a) {
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
  const TableEntry te = a.table[slot];
  copy_desc<Real>(g, &fx->wd, te.wd);
  g.sync();
  walker_steps<Real>(g, fx, base + fixed_bytes<Real>(), a, te.idx);
}

cudaError_t launch_run(const RunArgs &a, int fp64, cudaStream_t st) {
  const int threads = a.G * a.groups_per_cta;
  const int blocks = (a.nw + a.groups_per_cta - 1) / a.groups_per_cta;
  const size_t smem = (size_t)a.group_bytes * a.groups_per_cta;
  if (a.nw == 0) return cudaSuccess;
  cudaError_t e;
  if (fp64) {
    e = cudaFuncSetAttribute(k_run<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_run<double><<<blocks, threads, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_run<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_run<float><<<blocks, threads, smem, st>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- plain form
//
// Scratch kept in the walker's global jscratch buffer between launches:
// PlainScratch, then for each COORD CV its dCN/dx records (A list, B list).

template <typename Real>
struct PlainScratch {
  double s[kMaxCv];
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

// a1 for one walker; results to the walker's scratch.
template <typename Real>
__global__ void __launch_bounds__(256) k_plain_cv(const WalkerDev *wdp, const void *coords, const long long *coff,
                                                  int widx) {
  using R4 = typename Rec4<Real>::T;
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = cta_group<Real>();
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(smem);
  copy_desc<Real>(g, &fx->wd, wdp);
  g.sync();
  const WalkerDev &wd = fx->wd;
  R4 *xs = reinterpret_cast<R4 *>(smem + fixed_bytes<Real>());
  unsigned char *cnmem = reinterpret_cast<unsigned char *>(xs + 2 * wd.natoms);
  const R4 *xin = reinterpret_cast<const R4 *>(coords) + coff[widx];
  int bad = 0;
  for (int i = g.t; i < wd.natoms; i += g.G) {
    R4 p = xin[i];
    xs[i] = p;
    bad |= finite_rec<Real>(p) ? 0 : 1;
  }
  if (g.t == 0) fx->flags = 0;
  Real bv[1] = {(Real)bad};
  grp_sum<1>(g, bv, fx->red);
  g.sync();
  PlainScratch<Real> *ps = reinterpret_cast<PlainScratch<Real> *>(wd.jscratch);
  if (bv[0] != 0) {
    if (g.t == 0) {
      ps->bad = 1;
      ps->flags = ABP_WFLAG_NONFINITE;
    }
    return;
  }
  eval_cvs<Real>(g, fx, xs, cnmem);
  if (g.t == 0) {
    ps->bad = 0;
    ps->flags = fx->flags;
    for (int k = 0; k < kMaxCv; ++k) {
      ps->s[k] = fx->s[k];
      for (int q = 0; q < 3; ++q) ps->com_u[k][q] = fx->com_u[k][q];
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 3; ++q) ps->dih_g[k][a][q] = fx->dih_g[k][a][q];
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
  copy_desc<Real>(g, &fx->wd, wdp);
  g.sync();
  const PlainScratch<Real> *ps = reinterpret_cast<const PlainScratch<Real> *>(fx->wd.jscratch);
  if (ps->bad) return;
  if (g.t < kMaxCv) fx->s[g.t] = ps->s[g.t];
  g.sync();
  deposit_step<Real>(g, fx, step, log);
}

// a4 + a5 for one walker.
template <typename Real>
__global__ void __launch_bounds__(256) k_plain_force(const WalkerDev *wdp, void *forces, const long long *foff, int widx,
                                                     int mode, long long step, DevCounters *ctr) {
  using R4 = typename Rec4<Real>::T;
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = cta_group<Real>();
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(smem);
  copy_desc<Real>(g, &fx->wd, wdp);
  g.sync();
  const WalkerDev &wd = fx->wd;
  R4 *fs = reinterpret_cast<R4 *>(smem + fixed_bytes<Real>()) + wd.natoms;
  unsigned char *cnmem = reinterpret_cast<unsigned char *>(fs + wd.natoms);
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
      fx->s[k] = ps->s[k];
      for (int q = 0; q < 3; ++q) fx->com_u[k][q] = ps->com_u[k][q];
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 3; ++q) fx->dih_g[k][a][q] = ps->dih_g[k][a][q];
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
  interp_step<Real>(g, fx);
  scatter_forces<Real>(g, fx, fs, cnmem);
  for (int i = g.t; i < wd.natoms; i += g.G) {
    R4 f = fs[i];
    if (mode == ABP_FORCES_ACCUMULATE) {
      R4 o = fo[i];
      o.x += f.x;
      o.y += f.y;
      o.z += f.z;
      fo[i] = o;
    } else {
      fo[i] = make_rec<Real>(f.x, f.y, f.z, 0);
    }
  }
  write_state<Real>(g, fx, step);
}

template <typename Real>
static cudaError_t plain_one(const PlainArgs &a, int w, cudaStream_t st) {
  const WalkerDev *wd = a.wd_dev[w];
  const int T = a.threads;
  size_t smem = (size_t)fixed_bytes<Real>() + a.dyn_bytes[w];
  cudaError_t e;
  e = cudaFuncSetAttribute(k_plain_cv<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_plain_cv<Real><<<1, T, smem, st>>>(wd, a.coords, a.coff, w);
  if (a.deposit[w]) {
    size_t sm2 = (size_t)fixed_bytes<Real>();
    k_plain_deposit<Real><<<1, 256, sm2, st>>>(wd, a.step, a.log);
  }
  e = cudaFuncSetAttribute(k_plain_force<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
  for (int i = threadIdx.x; i < natoms; i += blockDim.x) {
    R4 f = src[i];
    if (mode == ABP_FORCES_ACCUMULATE) {
      R4 o = dst[i];
      o.x += f.x;
      o.y += f.y;
      o.z += f.z;
      dst[i] = o;
    } else {
      dst[i] = make_rec<Real>(f.x, f.y, f.z, 0);
    }
  }
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
