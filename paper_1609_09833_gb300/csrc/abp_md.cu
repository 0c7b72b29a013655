// abp_md.cu -- the closed-loop form (abp_md_run): the force call inside a
// model MD engine on the device, so that the coordinates of step t + 1 come
// from the bias force of step t without a host round trip (the biased MD
// cycle of the paper's Figure "cycle", with overdamped Langevin dynamics in
// place of GROMACS).
//
//   k_md   one warp per walker, for walkers whose CVs are COM distances,
//          dihedrals or RMSDs (the windowed form's walkers). A step is a
//          dependent chain -- a1, a2 + a3 on deposit steps, a4, a5, the move --
//          so a walker's steps cannot overlap one another; the warp keeps the
//          walker's atoms in shared memory for the whole launch and runs each
//          phase with the windowed form's per-step operations
//          (abp_window_ops.cuh): the same CVs, axis state, height, stencil
//          and interpolation arithmetic. The noise of a step is drawn while
//          its interpolation corners are in flight.
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

// Shared-memory layout of one walker's warp (bytes from the end of its
// GroupFixed): the atoms, the step's record, the potential's Jacobian
// factors, each atom's noise, the a5 term tables and the CV atom lists.
struct MdLayout {
  int xs, st, ju, nz, cnt, terms, lists, total;
};

__host__ __device__ inline MdLayout md_layout(int natoms, const CvDev *cv, int d, int fp64) {
  MdLayout L;
  const int rsz = fp64 ? 32 : 16, real = fp64 ? 8 : 4;
  int off = 0;
  L.xs = off;
  off += natoms * rsz;
  L.st = off;
  off += align32(fp64 ? (int)sizeof(StepRec<double>) : (int)sizeof(StepRec<float>));
  L.ju = off;
  off += align32(kMaxCv * 12 * real);
  L.nz = off;
  off += align16(natoms * 3 * real);
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

template <typename Real, int DIM, int UNR>
__global__ void __launch_bounds__(128) k_md(MdRunArgs a) {
  using R4 = typename Rec4<Real>::T;
  constexpr int NC = 1 << DIM;
  extern __shared__ __align__(32) unsigned char smem[];
  const RunArgs &ra = a.r;
  const int wpc = blockDim.x >> 5;  // walkers (warps) per CTA
  const int gid = threadIdx.x >> 5;
  const int slot = blockIdx.x * wpc + gid;
  if (slot >= ra.nw) return;  // a whole warp
  Grp g;
  g.G = 32;
  g.gid = gid;
  g.t = threadIdx.x & 31;
  g.lane = g.t;
  g.warp = 0;
  g.nwarps = 1;
  unsigned char *base = smem + (size_t)gid * ra.group_bytes;
  GroupFixed<Real> *fx = reinterpret_cast<GroupFixed<Real> *>(base);
  unsigned char *dyn = base + md_fixed_bytes<Real>();
  const TableEntry te = ra.table[slot];
  {
    const int *s = reinterpret_cast<const int *>(te.wd);
    int *d = reinterpret_cast<int *>(&fx->wd);
    for (int i = g.t; i < (int)(sizeof(WalkerDev) / 4); i += 32) d[i] = s[i];
  }
  __syncwarp();
  const WalkerDev &wd = fx->wd;
  const int natoms = wd.natoms;
  const MdLayout L = md_layout(natoms, wd.cv, DIM, sizeof(Real) == 8);
  {
    // the CV atom lists (and COM weights) into shared memory
    unsigned char *cur = dyn + L.lists;
    for (int k = 0; k < DIM; ++k) {
      const CvDev &c = wd.cv[k];
      int32_t *ia = reinterpret_cast<int32_t *>(cur);
      int32_t *ib = ia + c.na;
      for (int i = g.t; i < c.na; i += 32) ia[i] = c.ia[i];
      for (int i = g.t; i < c.nb; i += 32) ib[i] = c.ib[i];
      cur += align16((c.na + c.nb) * 4);
      Real *wa = nullptr, *wb = nullptr;
      if (c.type == ABP_CV_COM_DIST) {
        wa = reinterpret_cast<Real *>(cur);
        wb = wa + c.na;
        for (int i = g.t; i < c.na; i += 32) wa[i] = sizeof(Real) == 4 ? (Real)c.wa[i] : (Real)c.wa64[i];
        for (int i = g.t; i < c.nb; i += 32) wb[i] = sizeof(Real) == 4 ? (Real)c.wb[i] : (Real)c.wb64[i];
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
  __syncwarp();
  R4 *xs = reinterpret_cast<R4 *>(dyn + L.xs);
  StepRec<Real> &st = *reinterpret_cast<StepRec<Real> *>(dyn + L.st);
  Real(*ju)[12] = reinterpret_cast<Real(*)[12]>(dyn + L.ju);
  Real *nz = reinterpret_cast<Real *>(dyn + L.nz);
  int *cnt = reinterpret_cast<int *>(dyn + L.cnt);
  AtomTerm<Real> *terms = reinterpret_cast<AtomTerm<Real> *>(dyn + L.terms);
  build_atom_terms<Real>(g, fx, cnt, terms);
  R4 *cio = reinterpret_cast<R4 *>(const_cast<void *>(ra.coords)) + ra.coff[te.idx];
  for (int i = g.t; i < natoms; i += 32) xs[i] = cio[i];
  R4 *fout = ra.forces ? reinterpret_cast<R4 *>(ra.forces) + ra.foff[te.idx] : reinterpret_cast<R4 *>(wd.fbuf);
  const int fmode = ra.forces ? ra.mode : ABP_FORCES_OVERWRITE;
  R4 *tout = a.traj ? reinterpret_cast<R4 *>(a.traj) + a.toff[te.idx] : nullptr;
  const long long step0 = ra.step0;
  const Real c1 = (Real)a.md.c1, c2 = (Real)a.md.c2;
  const GroupLayout Lnone{};
  long long rem = step0 % wd.stride;
  long long next_dep = rem == 0 ? 0 : wd.stride - rem;
  int last = -1;  // the last step run
  __syncwarp();
  for (int t = 0; t < ra.nsteps; ++t) {
    const long long step = step0 + t;
    // the step's coordinates must be finite; a walker that meets non-finite
    // ones stops (its state says so)
    int bad = 0;
    for (int i = g.t; i < natoms; i += 32) bad |= finite_rec<Real>(xs[i]) ? 0 : 1;
    if (__any_sync(0xffffffffu, bad)) {
      if (g.t == 0) {
        wd.state->flags = ABP_WFLAG_NONFINITE;
        atomicAdd(&ra.ctr->nonfinite, 1);
      }
      break;
    }
    const bool dep = t == next_dep;
    if (dep) next_dep += wd.stride;
    // a1: every CV of the step into its record (COM distances on a lane pair,
    // the others on lane 0), then the step's flags
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      if (wd.cv[k].type == ABP_CV_COM_DIST)
        window_com2<Real>(fx, xs, k, dep, g.t < 2, g.t & 1, st);
      else if (g.t == 0)
        window_cv<Real>(fx, xs, k, dep, st);
    }
    __syncwarp();
    if (g.t == 0) {
      step_flags<Real>(DIM, dep, st);
      // the CV potential's factors: dU/ds_k times the CV's Jacobian factors
      Real sk[3] = {0, 0, 0}, dU[3];
#pragma unroll
      for (int k = 0; k < DIM; ++k) sk[k] = st.s[k];
      md_potential_grad<Real>(a.md, sk, dU);
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const int nj = wd.cv[k].type == ABP_CV_COM_DIST ? 3 : 12;
        for (int q = 0; q < nj; ++q) ju[k][q] = st.jac[k][q] * dU[k];
      }
    }
    __syncwarp();
    // a2 + a3 on a deposit step: height from the grid before the deposit,
    // then the stencil by the whole warp
    if (dep) {
      window_dep_axis<Real>(g, fx, st);
      __syncwarp();
      build_tables<Real>(g, fx);
      if (g.t == 0) window_height<Real, DIM>(fx, st, step, ra.log);
      __syncwarp();
      deposit_stencil<Real, false, UNR>(g, fx, Lnone, nullptr);
      __syncwarp();
    }
    // a4: lane 0 reads the corners; the warp draws the step's noise while
    // they are in flight
    float4 ca[NC], cb[NC];
    if (g.t == 0) interp_load<Real, DIM>(wd, st, ca, cb);
    for (int i = g.t; i < natoms; i += 32) {
      Real n3[3];
      md_normals(a.md.seed, te.stream, step, i, n3);
      nz[3 * i] = n3[0];
      nz[3 * i + 1] = n3[1];
      nz[3 * i + 2] = n3[2];
    }
    if (g.t == 0) interp_combine<Real, DIM>(wd, st, ca, cb);
    __syncwarp();
    // a5 and the move: each atom's bias force from its terms (as the
    // windowed form sums them: -sum_k dV_b/ds_k ds_k/dx), the potential's
    // force -sum_k dU/ds_k ds_k/dx from the same terms on the dU-scaled
    // factors, then x += c1 (F_bias + F_U) + c2 xi
    const bool keep_f = ra.forces || t == ra.nsteps - 1;
    for (int i = g.t; i < natoms; i += 32) {
      const AtomTerm<Real> *ti = terms + i * kAtomTerms;
      const int ne = cnt[i];
      const Real *J = &st.jac[0][0];
      const Real *JU = &ju[0][0];
      Real f0 = 0, f1 = 0, f2 = 0, u0 = 0, u1 = 0, u2 = 0;
      for (int q = 0; q < ne; ++q) {
        const Real w = ti[q].w;
        const Real *v = J + ti[q].off;
        const Real *vu = JU + ti[q].off;
        f0 += w * v[0];
        f1 += w * v[1];
        f2 += w * v[2];
        u0 += w * vu[0];
        u1 += w * vu[1];
        u2 += w * vu[2];
      }
      R4 x = xs[i];
      if (tout) tout[(long long)t * a.tstride + i] = x;
      if (keep_f) {
        R4 *fo = fout + (ra.forces ? (long long)t * ra.fstride : 0) + i;
        store_force<Real>(fo, make_rec<Real>(f0, f1, f2, 0), fmode);
      }
      x.x += c1 * (f0 + u0) + c2 * nz[3 * i];
      x.y += c1 * (f1 + u1) + c2 * nz[3 * i + 1];
      x.z += c1 * (f2 + u2) + c2 * nz[3 * i + 2];
      xs[i] = x;
    }
    last = t;
    __syncwarp();
  }
  // the moved atoms back to the caller, and the walker's state after its
  // last step
  for (int i = g.t; i < natoms; i += 32) cio[i] = xs[i];
  if (g.t == 0 && last >= 0) {
    WalkerState ws;
    for (int k = 0; k < 3; ++k) {
      ws.s[k] = k < DIM ? (double)st.s[k] + (double)st.sl[k] : 0.0;
      ws.dV[k] = k < DIM ? (double)st.dv[k] : 0.0;
    }
    ws.V = (double)st.V;
    ws.flags = st.flags;
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

cudaError_t launch_md(const MdRunArgs &a, int fp64, int dim, cudaStream_t st) {
  const RunArgs &r = a.r;
  if (r.nw == 0) return cudaSuccess;
  const int wpc = r.groups_per_cta;
  const int threads = 32 * wpc;
  const int blocks = (r.nw + wpc - 1) / wpc;
  const size_t smem = (size_t)r.group_bytes * wpc;
  void (*k)(MdRunArgs);
  if (fp64)
    k = dim == 1 ? k_md<double, 1, 4> : dim == 2 ? k_md<double, 2, 4> : k_md<double, 3, 4>;
  else
    k = dim == 1 ? k_md<float, 1, 7> : dim == 2 ? k_md<float, 2, 7> : k_md<float, 3, 7>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<blocks, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace abp
