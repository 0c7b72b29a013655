// abp_big.cu -- the phased form of the force call, for walkers that share a
// grid (multiple-walker runs) or that are too large for one shared-memory
// walker group. One MD step is five launches over all such walkers:
//
//   k_big_cn       a1, coordination numbers: the A x B pair sum split over
//                  CTAs by chunks of B (kBigChunk entries); each CTA writes
//                  dCN/dx of its B entries and its partial CN and A gradients
//   k_big_cvs      a1 (other CVs, partial sums combined in chunk order) and
//                  a2: every walker's hill height from the grid as it was
//                  before any deposit of the step (Jacobi order)
//   k_big_deposit  a3: the hills; shared grids add them to the FP64 shadow
//                  with atomics (order-independent up to FP64 rounding), own
//                  grids with the two-sum update of the fused form
//   k_big_refresh  shared grids: FP32 fields = FP64 shadow split into
//                  value + compensation (about 48 bits kept)
//   k_big_force    a4 + a5: interpolation after all deposits, chain rule
//
// FP32_COMP grids only. The paper's bias routine is the serial counterpart
// (one CPU rank), SI "Minimization of Interprocess Communications".
#include <cuda_runtime.h>

#include <vector>

#include "abp_device.cuh"
#include "abp_launch.h"
#include "abp_md.cuh"

namespace abp {

namespace {

constexpr int kBigThreads = 256;
constexpr int kBigJB = 4;
constexpr int kBigChunk = kBigThreads * kBigJB;
constexpr int kStencilPerBlock = 2048;

__host__ __device__ constexpr int fixed_bytes_f() { return (int)((sizeof(GroupFixed<float>) + 31) & ~(size_t)31); }

__host__ __device__ inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Per-walker scratch of the phased form (in the walker's jscratch):
//   BigHead | jA[na] | jB[nb] | part_s[nchunk][2] | part_g[nchunk][na][3]
// for the walker's (single) COORD CV; jA/jB hold dCN/dx per list entry.
struct BigHead {
  float sh[kMaxCv], sl[kMaxCv];
  float com_u[kMaxCv][3];
  float dih_g[kMaxCv][4][3];
  int da[kMaxCv], dc[kMaxCv], ic_log[kMaxCv];
  float df[kMaxCv];
  float hf;
  int dep, bad, flags;
  double h;
};

__host__ __device__ inline int big_cn_index(const WalkerDev &wd) {
  for (int k = 0; k < wd.g.d; ++k)
    if (wd.cv[k].type == ABP_CV_COORD) return k;
  return -1;
}

__host__ __device__ inline int big_nchunks(const WalkerDev &wd) {
  int k = big_cn_index(wd);
  return k < 0 ? 0 : (wd.cv[k].nb + kBigChunk - 1) / kBigChunk;
}

struct BigLayout {
  size_t head, jA, jB, part_s, part_g, terms, nterm, total;
};

__host__ __device__ inline BigLayout big_layout(const WalkerDev &wd) {
  BigLayout L;
  int k = big_cn_index(wd);
  int na = k < 0 ? 0 : wd.cv[k].na, nb = k < 0 ? 0 : wd.cv[k].nb;
  int nc = big_nchunks(wd);
  L.head = 0;
  L.jA = up256(sizeof(BigHead));
  L.jB = L.jA + (size_t)na * 16;
  L.part_s = up256(L.jB + (size_t)nb * 16);
  L.part_g = up256(L.part_s + (size_t)nc * 8);
  // per atom, its a5 terms (big_atom_terms) and their count
  L.terms = up256(L.part_g + (size_t)nc * na * 12);
  L.nterm = up256(L.terms + (size_t)wd.natoms * kAtomTerms * 4);
  L.total = up256(L.nterm + (size_t)wd.natoms);
  return L;
}

// Term codes of the force phase: kind | k << 3 | list position << 5.
enum { kTermComA = 0, kTermComB = 1, kTermDih = 2, kTermCnA = 3, kTermCnB = 4 };

int big_atom_terms(const WalkerDev &hd, const abp_walker_desc *d, std::vector<int32_t> &terms,
                   std::vector<uint8_t> &cnt) {
  const int n = hd.natoms;
  terms.assign((size_t)n * kAtomTerms, 0);
  cnt.assign((size_t)n, 0);
  auto add = [&](int atom, int kind, int k, int pos) -> int {
    if (atom < 0 || atom >= n || cnt[atom] >= kAtomTerms || pos >= (1 << 26)) return -1;
    terms[(size_t)atom * kAtomTerms + cnt[atom]] = kind | (k << 3) | (pos << 5);
    cnt[atom] += 1;
    return 0;
  };
  // CV by CV, list A before list B: the order in which a5 adds them
  for (int k = 0; k < hd.g.d; ++k) {
    const abp_cv_desc &c = d->cv[k];
    const bool com = c.type == ABP_CV_COM_DIST, cn = c.type == ABP_CV_COORD;
    if (!com && !cn && c.type != ABP_CV_DIHEDRAL) return -1;
    const int na = c.type == ABP_CV_DIHEDRAL ? 4 : c.n_a;
    for (int i = 0; i < na; ++i)
      if (add(c.idx_a[i], com ? kTermComA : cn ? kTermCnA : kTermDih, k, i)) return -1;
    if (com || cn)
      for (int i = 0; i < c.n_b; ++i)
        if (add(c.idx_b[i], com ? kTermComB : kTermCnB, k, i)) return -1;
  }
  return 0;
}

size_t big_scratch_bytes(const WalkerDev &hd) { return big_layout(hd).total; }
size_t big_terms_offset(const WalkerDev &hd) { return big_layout(hd).terms; }
size_t big_nterm_offset(const WalkerDev &hd) { return big_layout(hd).nterm; }
int big_cn_count(const WalkerDev &hd) {
  int n = 0;
  for (int k = 0; k < hd.g.d; ++k) n += hd.cv[k].type == ABP_CV_COORD;
  return n;
}
int big_chunks(const WalkerDev &hd) { return big_nchunks(hd); }

// ---------------------------------------------------------------- k_big_cn

// Minimum image d - L rint(d / L) with rint formed on the FMA pipe: adding
// and subtracting 1.5 2^23 rounds d / L to the nearest integer exactly for
// |d / L| < 2^22 (ties go to even, where either image has the same length).
__device__ __forceinline__ float min_image_rn(float d, float L, float invL) {
  const float M = 12582912.0f;
  const float t = __fsub_rn(__fmaf_rn(d, invL, M), M);
  return __fmaf_rn(-L, t, d);
}

// The A gradients of one block (4 A atoms x 3 components, this lane's part)
// summed over the warp by a reduce-scatter: the half-warps exchange half of
// the values (atoms 0, 1 | 2, 3), then the quarter-warps (one atom each),
// then three butterfly levels over the remaining three; lane 8 q holds atom
// q's sums, which it adds to the warp's accumulators.
__device__ __forceinline__ void reduce_block_grads(const float (&gi)[4][3], int lane, int i0, int na, float *mylig) {
  const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
  float w6[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const float lo = gi[j / 3][j % 3], hi = gi[2 + j / 3][j % 3];
    const float send = h16 ? lo : hi;
    w6[j] = (h16 ? hi : lo) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float w3[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float send = h8 ? w6[j] : w6[3 + j];
    w3[j] = (h8 ? w6[3 + j] : w6[j]) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1)
#pragma unroll
    for (int j = 0; j < 3; ++j) w3[j] += __shfl_xor_sync(0xffffffffu, w3[j], o);
  const int ii = (h16 ? 2 : 0) + (h8 ? 1 : 0);
  if ((lane & 7) == 0 && i0 + ii < na)
#pragma unroll
    for (int q = 0; q < 3; ++q) mylig[(i0 + ii) * 3 + q] += w3[q];
}

// One CTA: the A x (one chunk of B) pairs of one walker's CN.
__global__ void __launch_bounds__(kBigThreads) k_big_cn(const BigItem *items, const void *coords,
                                                        const long long *coff, long long step_off) {
  extern __shared__ __align__(32) unsigned char smem[];
  const BigItem it = items[blockIdx.x];
  const WalkerDev *wd = it.wd;
  const int k = big_cn_index(*wd);
  const CvDev &c = wd->cv[k];
  const int na = c.na, nb = c.nb;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = kBigThreads / 32;
  const float4 *x = reinterpret_cast<const float4 *>(coords) + coff[it.widx] + step_off;
  float4 *As = reinterpret_cast<float4 *>(smem);
  float *lig = reinterpret_cast<float *>(As + na);  // [nwarps][na][3]
  for (int i = t; i < na; i += kBigThreads) As[i] = x[c.ia[i]];
  for (int q = t; q < nwarps * na * 3; q += kBigThreads) lig[q] = 0.f;
  __syncthreads();
  const float k2 = (float)c.inv_r0sq, c6 = -6.f * k2;
  const bool pbc = c.pbc != 0;
  const float bx = (float)c.box[0], by = (float)c.box[1], bz = (float)c.box[2];
  const float ibx = (float)c.inv_box[0], iby = (float)c.inv_box[1], ibz = (float)c.inv_box[2];
  const int j0 = it.chunk * kBigChunk;
  float xj[kBigJB], yj[kBigJB], zj[kBigJB], gxj[kBigJB], gyj[kBigJB], gzj[kBigJB], mj[kBigJB];
#pragma unroll
  for (int jj = 0; jj < kBigJB; ++jj) {
    int j = j0 + jj * kBigThreads + t;
    bool ok = j < nb;
    float4 p = x[c.ib[ok ? j : 0]];
    xj[jj] = p.x;
    yj[jj] = p.y;
    zj[jj] = p.z;
    mj[jj] = ok ? 1.f : 0.f;
    gxj[jj] = gyj[jj] = gzj[jj] = 0.f;
  }
  // the thread's CN terms: each block of 4 A atoms x kBigJB B entries summed
  // in (A, B) order, the block's sum added to a compensated (two-sum)
  // accumulator
  float sacc = 0.f, scomp = 0.f;
  float *mylig = lig + warp * na * 3;
  // every B entry of this CTA in range: blocks of 4 A atoms need no mask
  // (a mask of 1 would change no bit)
  const bool fullj = j0 + kBigJB * kBigThreads <= nb;
  for (int i0 = 0; i0 < na; i0 += 4) {
    float gi[4][3];
    float part = 0.f;
    if (fullj && i0 + 4 <= na) {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        gi[ii][0] = gi[ii][1] = gi[ii][2] = 0.f;
        float4 a = As[i0 + ii];
#pragma unroll
        for (int jj = 0; jj < kBigJB; ++jj) {
          float dx = a.x - xj[jj], dy = a.y - yj[jj], dz = a.z - zj[jj];
          if (pbc) {
            dx = min_image_rn(dx, bx, ibx);
            dy = min_image_rn(dy, by, iby);
            dz = min_image_rn(dz, bz, ibz);
          }
          float q = (dx * dx + dy * dy + dz * dz) * k2;
          float q2 = q * q;
          float sw = __fdividef(1.f, 1.f + q2 * q);
          part += sw;
          float gf = c6 * q2 * sw * sw;
          gi[ii][0] += gf * dx;
          gi[ii][1] += gf * dy;
          gi[ii][2] += gf * dz;
          gxj[jj] -= gf * dx;
          gyj[jj] -= gf * dy;
          gzj[jj] -= gf * dz;
        }
      }
    } else {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        gi[ii][0] = gi[ii][1] = gi[ii][2] = 0.f;
        int i = i0 + ii;
        bool oki = i < na;
        float4 a = As[oki ? i : 0];
#pragma unroll
        for (int jj = 0; jj < kBigJB; ++jj) {
          float dx = a.x - xj[jj], dy = a.y - yj[jj], dz = a.z - zj[jj];
          if (pbc) {
            dx = min_image_rn(dx, bx, ibx);
            dy = min_image_rn(dy, by, iby);
            dz = min_image_rn(dz, bz, ibz);
          }
          float q = (dx * dx + dy * dy + dz * dz) * k2;
          float q2 = q * q;
          float sw = __fdividef(1.f, 1.f + q2 * q);
          float m = oki ? mj[jj] : 0.f;
          part += m * sw;
          float gf = c6 * m * q2 * sw * sw;
          gi[ii][0] += gf * dx;
          gi[ii][1] += gf * dy;
          gi[ii][2] += gf * dz;
          gxj[jj] -= gf * dx;
          gyj[jj] -= gf * dy;
          gzj[jj] -= gf * dz;
        }
      }
    }
    {
      float tsum, terr;
      two_sum<float>(sacc, part, tsum, terr);
      sacc = tsum;
      scomp += terr;
    }
    reduce_block_grads(gi, lane, i0, na, mylig);
  }
  unsigned char *js = reinterpret_cast<unsigned char *>(wd->jscratch);
  const BigLayout L = big_layout(*wd);
  float4 *jB = reinterpret_cast<float4 *>(js + L.jB);
#pragma unroll
  for (int jj = 0; jj < kBigJB; ++jj) {
    int j = j0 + jj * kBigThreads + t;
    if (j < nb) jB[j] = make_float4(gxj[jj], gyj[jj], gzj[jj], 0.f);
  }
  // this chunk's CN as hi + lo: warps in order, lanes by butterfly
  float sh, sl;
  two_sum<float>(sacc, scomp, sh, sl);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
    ff_add<float>(sh, sl, oh, ol);
  }
  // (every lane now holds the same pair: the pairwise add is commutative)
  __shared__ float wsum[kBigThreads / 32][2];
  if (lane == 0) {
    wsum[warp][0] = sh;
    wsum[warp][1] = sl;
  }
  __syncthreads();
  float *part_s = reinterpret_cast<float *>(js + L.part_s) + 2 * it.chunk;
  if (t == 0) {
    float h = wsum[0][0], l = wsum[0][1];
    for (int w = 1; w < nwarps; ++w) ff_add<float>(h, l, wsum[w][0], wsum[w][1]);
    part_s[0] = h;
    part_s[1] = l;
  }
  float *part_g = reinterpret_cast<float *>(js + L.part_g) + (size_t)it.chunk * na * 3;
  for (int q = t; q < na * 3; q += kBigThreads) {
    float acc = 0.f;
    for (int w = 0; w < nwarps; ++w) acc += lig[w * na * 3 + q];
    part_g[q] = acc;
  }
}

// ---------------------------------------------------------------- k_big_cvs

__device__ __forceinline__ Grp big_group() {
  Grp g;
  g.G = blockDim.x;
  g.gid = 0;
  g.t = threadIdx.x;
  g.lane = threadIdx.x & 31;
  g.warp = threadIdx.x >> 5;
  g.nwarps = blockDim.x >> 5;
  return g;
}

__device__ void big_load_desc(const Grp &g, GroupFixed<float> *fx, const WalkerDev *wdp) {
  const int *s = reinterpret_cast<const int *>(wdp);
  int *d = reinterpret_cast<int *>(&fx->wd);
  for (int i = g.t; i < (int)(sizeof(WalkerDev) / 4); i += g.G) d[i] = s[i];
  g.sync();
  if (g.t < kMaxCv) {
    const CvDev &c = fx->wd.cv[g.t];
    fx->ia[g.t] = c.ia;
    fx->ib[g.t] = c.ib;
    fx->wa[g.t] = c.wa;
    fx->wb[g.t] = c.wb;
  }
  if (g.t == 0) {
    fx->flags = 0;
    fx->clamped = 0;
  }
  g.sync();
}

// Centre-of-mass distance with compensated arithmetic: each weighted offset
// w (x - r_G) is split exactly into hi + lo (the difference by two_sum, the
// product's error by fma; w times the difference's low part, tiny, rounded
// once), summed as hi + lo pairs, and |d| is taken in hi + lo. Groups spread
// over a large box (as a group of environment atoms is) otherwise lose the
// ~1e-8 relative accuracy a hill a few grid spacings wide needs.
__device__ void cv_com_ff(const Grp &g, GroupFixed<float> *fx, int k, const float4 *xs) {
  const CvDev &c = fx->wd.cv[k];
  const float4 ra = xs[c.ia[0]], rb = xs[c.ib[0]];
  float h[6] = {0, 0, 0, 0, 0, 0}, l[6] = {0, 0, 0, 0, 0, 0};
  auto acc = [&](int q, float w, float x, float r) {
    float dh, dl;
    two_sum<float>(x, -r, dh, dl);  // x - r exactly
    float p = __fmul_rn(w, dh);
    float e = __fmaf_rn(w, dl, __fmaf_rn(w, dh, -p));
    ff_add<float>(h[q], l[q], p, e);
  };
  for (int i = g.t; i < c.na; i += g.G) {
    float w = c.wa[i];
    float4 p = xs[c.ia[i]];
    acc(0, w, p.x, ra.x);
    acc(1, w, p.y, ra.y);
    acc(2, w, p.z, ra.z);
  }
  for (int i = g.t; i < c.nb; i += g.G) {
    float w = c.wb[i];
    float4 p = xs[c.ib[i]];
    acc(3, w, p.x, rb.x);
    acc(4, w, p.y, rb.y);
    acc(5, w, p.z, rb.z);
  }
  for (int q = 0; q < 6; ++q) grp_sum_ff<float>(g, h[q], l[q], fx->red);
  if (g.t != 0) return;
  // equal masses: the weights' FP32 rounding, one factor per group
  for (int q = 0; q < 3; ++q) {
    if (c.wc_a != 0.f) ff_add<float>(h[q], l[q], __fmul_rn(h[q], c.wc_a), 0.f);
    if (c.wc_b != 0.f) ff_add<float>(h[3 + q], l[3 + q], __fmul_rn(h[3 + q], c.wc_b), 0.f);
  }
  float dh[3], dl[3];
  const float ra3[3] = {ra.x, ra.y, ra.z}, rb3[3] = {rb.x, rb.y, rb.z};
  for (int q = 0; q < 3; ++q) {
    float rdh, rdl;  // r_B - r_A exactly, as hi + lo
    two_sum<float>(rb3[q], -ra3[q], rdh, rdl);
    float s, e;
    two_sum<float>(rdh, h[3 + q], s, e);
    e += l[3 + q] + rdl;
    float s2, e2;
    two_sum<float>(s, -h[q], s2, e2);
    e2 += e - l[q];
    dh[q] = s2 + e2;
    dl[q] = e2 - (dh[q] - s2);
    if (c.pbc) {
      float shift = (float)c.box[q] * floor(dh[q] * (float)c.inv_box[q] + 0.5f);
      float t, te;
      two_sum<float>(dh[q], -shift, t, te);
      dh[q] = t;
      dl[q] += te;
    }
  }
  // r^2 = sum (dh + dl)^2 in hi + lo, then r = sqrt with one Newton correction
  float r2h = 0, r2l = 0;
  for (int q = 0; q < 3; ++q) {
    float p = dh[q] * dh[q];
    float e = fmaf(dh[q], dh[q], -p) + 2.f * dh[q] * dl[q];
    ff_add<float>(r2h, r2l, p, e);
  }
  float rh = sqrtf(r2h);
  float rl = rh > 0 ? (fmaf(-rh, rh, r2h) + r2l) / (2.f * rh) : 0.f;
  fx->sh[k] = rh;
  fx->sl[k] = rl;
  if (rh > 0) {
    float ir = 1.f / rh;
    for (int q = 0; q < 3; ++q) fx->com_u[k][q] = dh[q] * ir;
  } else {
    for (int q = 0; q < 3; ++q) fx->com_u[k][q] = 0;
    fx->flags |= ABP_WFLAG_SINGULAR;
  }
}

// One CTA per walker: CVs, axis state, height; hill record to the head.
__global__ void __launch_bounds__(kBigThreads) k_big_cvs(const BigItem *walkers, const void *coords,
                                                         const long long *coff, long long step_off, long long step,
                                                         DepositLog log, DevCounters *ctr) {
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = big_group();
  GroupFixed<float> *fx = reinterpret_cast<GroupFixed<float> *>(smem);
  const BigItem it = walkers[blockIdx.x];
  big_load_desc(g, fx, it.wd);
  const WalkerDev &wd = fx->wd;
  const float4 *x = reinterpret_cast<const float4 *>(coords) + coff[it.widx] + step_off;
  unsigned char *js = reinterpret_cast<unsigned char *>(wd.jscratch);
  BigHead *head = reinterpret_cast<BigHead *>(js);
  int bad = 0;
  for (int i = g.t; i < wd.natoms; i += g.G) {
    float4 p = x[i];
    bad |= (isfinite(p.x) && isfinite(p.y) && isfinite(p.z)) ? 0 : 1;
  }
  if (grp_any<float>(g, fx, bad)) {
    if (g.t == 0) {
      head->bad = 1;
      head->dep = 0;
      head->flags = ABP_WFLAG_NONFINITE;
      atomicAdd(&ctr->nonfinite, 1);
    }
    return;
  }
  const BigLayout L = big_layout(wd);
  const int kc = big_cn_index(wd);
  for (int k = 0; k < wd.g.d; ++k) {
    const CvDev &c = wd.cv[k];
    if (c.type == ABP_CV_COM_DIST) {
      cv_com_ff(g, fx, k, x);
    } else if (c.type == ABP_CV_DIHEDRAL) {
      cv_dihedral<float>(g, fx, k, x);
    }
  }
  if (kc >= 0) {
    const CvDev &c = wd.cv[kc];
    const int nc = big_nchunks(wd);
    const float *part_s = reinterpret_cast<const float *>(js + L.part_s);
    const float *part_g = reinterpret_cast<const float *>(js + L.part_g);
    if (g.t == 0) {
      float h = part_s[0], l = part_s[1];
      for (int q = 1; q < nc; ++q) ff_add<float>(h, l, part_s[2 * q], part_s[2 * q + 1]);
      fx->sh[kc] = h;
      fx->sl[kc] = l;
    }
    float4 *jA = reinterpret_cast<float4 *>(js + L.jA);
    for (int i = g.t; i < c.na; i += g.G) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      for (int q = 0; q < nc; ++q) {
        const float *p = part_g + ((size_t)q * c.na + i) * 3;
        a0 += p[0];
        a1 += p[1];
        a2 += p[2];
      }
      jA[i] = make_float4(a0, a1, a2, 0.f);
    }
  }
  g.sync();
  const bool dep = (step % wd.stride) == 0;
  if (g.t < wd.g.d) axis_setup<float>(fx, g.t, dep);
  g.sync();
  if (dep && g.warp == 0) {
    // V_b(s_t) before this step's deposits: the FP64 shadow of a shared
    // grid, the value + compensation records of an own grid
    const GridDev &gd = wd.g;
    double acc = 0;
    if (g.lane < (1 << gd.d)) {
      double w = 1;
      long long node = 0, mul = 1;
      for (int k = 0; k < gd.d; ++k) {
        int hi = (g.lane >> k) & 1;
        double f = (double)fx->f[k];
        w *= hi ? f : 1.0 - f;
        node += mul * (hi ? fx->i1[k] : fx->i0[k]);
        mul *= gd.n[k];
      }
      double v;
      node = chk_node(gd, node);
      if (gd.shared) {
        v = gd.shadow[node * 4];
      } else {
        double vv[4];
        rec_values<double>(gd, reinterpret_cast<const unsigned char *>(gd.rec) + node * gd.rec_bytes, vv);
        v = vv[0];
      }
      acc = w * v;
    }
    for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (g.lane == 0) {
      double h = wd.w * exp(-acc * wd.inv_dT);
      head->h = h;
      head->hf = (float)h;
      if (log.rec) {
        unsigned long long slot = atomicAdd(log.count, 1ull);
        if (slot < log.cap) {
          abp_deposit_rec r;
          r.step = step;
          r.walker_id = wd.id;
          for (int k = 0; k < 3; ++k) {
            r.ic[k] = k < gd.d ? fx->ic_log[k] : 0;
            r.s[k] = k < gd.d ? (double)fx->sh[k] + (double)fx->sl[k] : 0.0;
          }
          r.height = h;
          log.rec[slot] = r;
        }
      }
    }
  }
  if (g.t == 0) {
    head->bad = 0;
    head->dep = dep ? 1 : 0;
    head->flags = fx->flags | (dep ? ABP_WFLAG_DEPOSIT : 0);
    for (int k = 0; k < kMaxCv; ++k) {
      head->sh[k] = fx->sh[k];
      head->sl[k] = fx->sl[k];
      head->da[k] = fx->da[k];
      head->dc[k] = fx->dc[k];
      head->df[k] = fx->df[k];
      head->ic_log[k] = fx->ic_log[k];
      for (int q = 0; q < 3; ++q) head->com_u[k][q] = fx->com_u[k][q];
      for (int a = 0; a < 4; ++a)
        for (int q = 0; q < 3; ++q) head->dih_g[k][a][q] = fx->dih_g[k][a][q];
    }
  }
}

// ---------------------------------------------------------------- deposit + refresh

// Stencil tables from the hill record (all CTAs of a walker build the same).
__device__ bool big_tables(const Grp &g, GroupFixed<float> *fx, const BigItem &it) {
  big_load_desc(g, fx, it.wd);
  const BigHead *head = reinterpret_cast<const BigHead *>(fx->wd.jscratch);
  if (!head->dep || head->bad) return false;
  if (g.t < kMaxCv) {
    fx->da[g.t] = head->da[g.t];
    fx->dc[g.t] = head->dc[g.t];
    fx->df[g.t] = head->df[g.t];
  }
  if (g.t == 0) fx->hf = head->hf;
  g.sync();
  build_tables<float>(g, fx);
  g.sync();
  return true;
}

__global__ void __launch_bounds__(kBigThreads) k_big_deposit(const BigItem *walkers) {
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = big_group();
  GroupFixed<float> *fx = reinterpret_cast<GroupFixed<float> *>(smem);
  if (!big_tables(g, fx, walkers[blockIdx.x])) return;
  const WalkerDev &wd = fx->wd;
  const GridDev &gd = wd.g;
  const int d = gd.d;
  const int s0 = 2 * wd.R[0] + 1, s1 = d > 1 ? 2 * wd.R[1] + 1 : 1, s2 = d > 2 ? 2 * wd.R[2] + 1 : 1;
  const int total = s0 * s1 * s2;
  const int first = blockIdx.y * kStencilPerBlock, last = min(total, first + kStencilPerBlock);
  const long long n0 = gd.n[0], n01 = n0 * (d > 1 ? gd.n[1] : 1);
  const float h = fx->hf;
  for (int idx = first + g.t; idx < last; idx += g.G) {
    int o0 = idx % s0, r = idx / s0, o1 = r % s1, o2 = r / s1;
    int j0 = fx->tabJ[0][o0];
    int j1 = d > 1 ? fx->tabJ[1][o1] : 0;
    int j2 = d > 2 ? fx->tabJ[2][o2] : 0;
    if ((j0 | j1 | j2) < 0) continue;
    float G = h * fx->tabG[0][o0];
    if (d > 1) G = G * fx->tabG[1][o1];
    if (d > 2) G = G * fx->tabG[2][o2];
    float d0 = fx->tabD[0][o0], d1 = d > 1 ? fx->tabD[1][o1] : 0.f, d2 = d > 2 ? fx->tabD[2][o2] : 0.f;
    const long long node = chk_node(gd, j0 + n0 * j1 + n01 * j2);
    if (gd.shared) {
      double *p = gd.shadow + node * 4;
      atomicAdd(p, (double)G);
      atomicAdd(p + 1, (double)__fmul_rn(G, d0));
      if (d > 1) atomicAdd(p + 2, (double)__fmul_rn(G, d1));
      if (d > 2) atomicAdd(p + 3, (double)__fmul_rn(G, d2));
    } else {
      rmw_node<float>(gd, reinterpret_cast<unsigned char *>(gd.rec) + node * gd.rec_bytes, G, d0, d1, d2);
    }
  }
}

__global__ void __launch_bounds__(kBigThreads) k_big_refresh(const BigItem *walkers) {
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = big_group();
  GroupFixed<float> *fx = reinterpret_cast<GroupFixed<float> *>(smem);
  if (!big_tables(g, fx, walkers[blockIdx.x])) return;
  const WalkerDev &wd = fx->wd;
  const GridDev &gd = wd.g;
  if (!gd.shared) return;
  const int d = gd.d;
  const int s0 = 2 * wd.R[0] + 1, s1 = d > 1 ? 2 * wd.R[1] + 1 : 1, s2 = d > 2 ? 2 * wd.R[2] + 1 : 1;
  const int total = s0 * s1 * s2;
  const int first = blockIdx.y * kStencilPerBlock, last = min(total, first + kStencilPerBlock);
  const long long n0 = gd.n[0], n01 = n0 * (d > 1 ? gd.n[1] : 1);
  for (int idx = first + g.t; idx < last; idx += g.G) {
    int o0 = idx % s0, r = idx / s0, o1 = r % s1, o2 = r / s1;
    int j0 = fx->tabJ[0][o0];
    int j1 = d > 1 ? fx->tabJ[1][o1] : 0;
    int j2 = d > 2 ? fx->tabJ[2][o2] : 0;
    if ((j0 | j1 | j2) < 0) continue;
    const long long node = chk_node(gd, j0 + n0 * j1 + n01 * j2);
    const double *p = gd.shadow + node * 4;
    float hi[4], lo[4];
    for (int q = 0; q < 4; ++q) {
      double v = q <= d ? p[q] : 0.0;
      hi[q] = (float)v;
      lo[q] = (float)(v - (double)hi[q]);
    }
    if (d == 1) {
      *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(gd.rec) + node * 16) =
          make_float4(hi[0], hi[1], lo[0], lo[1]);
    } else {
      float4 *q = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(gd.rec) + node * 32);
      q[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
      q[1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// ---------------------------------------------------------------- k_big_force

// a4 + a5 of one walker's atoms [blockIdx.x * kBigThreads, + kBigThreads):
// each CTA forms the walker's dV/ds (a few corner reads), then each thread
// sums its atom's terms in the walker's fixed order (CV by CV, list A before
// list B) and writes the walker's force buffer and, when given, the
// caller's.
__global__ void __launch_bounds__(kBigThreads) k_big_force(const BigItem *walkers, void *forces,
                                                           const long long *foff, long long force_step_off, int mode,
                                                           long long step) {
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = big_group();
  GroupFixed<float> *fx = reinterpret_cast<GroupFixed<float> *>(smem);
  const BigItem it = walkers[blockIdx.y];
  const int i0 = blockIdx.x * kBigThreads;
  if (i0 >= it.wd->natoms) return;  // the whole CTA: past this walker's atoms
  big_load_desc(g, fx, it.wd);
  const WalkerDev &wd = fx->wd;
  unsigned char *js = reinterpret_cast<unsigned char *>(wd.jscratch);
  const BigHead *head = reinterpret_cast<const BigHead *>(js);
  float4 *fb = reinterpret_cast<float4 *>(wd.fbuf);
  float4 *fo = forces ? reinterpret_cast<float4 *>(forces) + foff[it.widx] + force_step_off : fb;
  const int fmode = forces ? mode : ABP_FORCES_OVERWRITE;
  const int i = i0 + g.t;
  if (head->bad) {
    if (fmode == ABP_FORCES_OVERWRITE && i < wd.natoms) fo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (blockIdx.x == 0 && g.t == 0) wd.state->flags = ABP_WFLAG_NONFINITE;
    return;
  }
  if (g.t < kMaxCv) {
    fx->sh[g.t] = head->sh[g.t];
    fx->sl[g.t] = head->sl[g.t];
    for (int q = 0; q < 3; ++q) fx->com_u[g.t][q] = head->com_u[g.t][q];
    for (int a = 0; a < 4; ++a)
      for (int q = 0; q < 3; ++q) fx->dih_g[g.t][a][q] = head->dih_g[g.t][a][q];
  }
  if (g.t == 0) fx->flags = head->flags;
  g.sync();
  if (g.t < wd.g.d) axis_setup<float>(fx, g.t, false);
  g.sync();
  GroupLayout Ldummy{};
  interp_step<float, false>(g, fx, Ldummy, nullptr);
  if (i < wd.natoms) {
    const BigLayout L = big_layout(wd);
    const int32_t *tt = reinterpret_cast<const int32_t *>(js + L.terms) + (size_t)i * kAtomTerms;
    const int ne = js[L.nterm + i];
    const float4 *jA = reinterpret_cast<const float4 *>(js + L.jA);
    const float4 *jB = reinterpret_cast<const float4 *>(js + L.jB);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    for (int q = 0; q < ne; ++q) {
      const int code = tt[q], kind = code & 7, k = (code >> 3) & 3, pos = code >> 5;
      const float dv = fx->dvds[k];
      if (kind == kTermComA || kind == kTermComB) {
        const float ux = fx->com_u[k][0] * dv, uy = fx->com_u[k][1] * dv, uz = fx->com_u[k][2] * dv;
        if (kind == kTermComA) {
          const float w = wd.cv[k].wa[pos];
          f0 += w * ux;
          f1 += w * uy;
          f2 += w * uz;
        } else {
          const float w = wd.cv[k].wb[pos];
          f0 -= w * ux;
          f1 -= w * uy;
          f2 -= w * uz;
        }
      } else if (kind == kTermDih) {
        f0 -= dv * fx->dih_g[k][pos][0];
        f1 -= dv * fx->dih_g[k][pos][1];
        f2 -= dv * fx->dih_g[k][pos][2];
      } else {
        const float4 j = kind == kTermCnA ? jA[pos] : jB[pos];
        f0 -= dv * j.x;
        f1 -= dv * j.y;
        f2 -= dv * j.z;
      }
    }
    fb[i] = make_float4(f0, f1, f2, 0.f);
    if (fo != fb) {
      if (fmode == ABP_FORCES_ACCUMULATE) {
        float4 o = fo[i];
        o.x += f0;
        o.y += f1;
        o.z += f2;
        fo[i] = o;
      } else {
        fo[i] = make_float4(f0, f1, f2, 0.f);
      }
    }
  }
  if (blockIdx.x == 0 && g.t == 0) {
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
}

// ---------------------------------------------------------------- k_big_move

// Closed loop (abp_md_run): after the force phase, the move of one walker's
// atoms [blockIdx.x * kBigThreads, + kBigThreads): x += c1 F_bias + c2 xi
// (this form takes no CV potential), the coordinates before the move to the
// trajectory records when given. A walker whose step saw non-finite
// coordinates does not move.
__global__ void __launch_bounds__(kBigThreads) k_big_move(const BigItem *walkers, MdParams md, void *xio,
                                                          const long long *coff, void *traj, const long long *toff,
                                                          long long traj_step_off, long long step) {
  const BigItem it = walkers[blockIdx.y];
  const WalkerDev *wd = it.wd;
  const int i = blockIdx.x * kBigThreads + threadIdx.x;
  if (i >= wd->natoms) return;
  const BigHead *head = reinterpret_cast<const BigHead *>(wd->jscratch);
  if (head->bad) return;
  float4 *x = reinterpret_cast<float4 *>(xio) + coff[it.widx] + i;
  const float4 f = reinterpret_cast<const float4 *>(wd->fbuf)[i];
  float4 p = *x;
  if (traj) reinterpret_cast<float4 *>(traj)[toff[it.widx] + traj_step_off + i] = p;
  float n[3];
  md_normals(md.seed, it.stream, step, i, n);
  const float c1 = (float)md.c1, c2 = (float)md.c2;
  p.x += c1 * f.x + c2 * n[0];
  p.y += c1 * f.y + c2 * n[1];
  p.z += c1 * f.z + c2 * n[2];
  *x = p;
}

// ---------------------------------------------------------------- launcher

cudaError_t launch_big_step(const BigArgs &a, cudaStream_t st) {
  const size_t fixed = (size_t)fixed_bytes_f();
  const int ph = a.phases ? a.phases : 31;
  LaunchTimer *tm = a.timer;
  auto t0 = [&](const char *k) {
    nvtxRangePushA(k);
    if (tm) tm->begin(k, st);
  };
  auto t1 = [&](const char *k) {
    if (tm) tm->end(k, st);
    nvtxRangePop();
  };
  cudaError_t e;
  if ((ph & 1) && a.ncn_items > 0) {
    e = smem_attr(reinterpret_cast<const void *>(k_big_cn), a.cn_smem);
    if (e != cudaSuccess) return e;
    t0("k_big_cn");
    k_big_cn<<<a.ncn_items, kBigThreads, a.cn_smem, st>>>(a.cn_items, a.coords, a.coff, a.step_off);
    t1("k_big_cn");
  }
  if (ph & 2) {
    t0("k_big_cvs");
    k_big_cvs<<<a.nw, kBigThreads, fixed, st>>>(a.walkers, a.coords, a.coff, a.step_off, a.step, a.log, a.ctr);
    t1("k_big_cvs");
  }
  dim3 grid(a.nw, (a.max_stencil + kStencilPerBlock - 1) / kStencilPerBlock);
  if (ph & 4) {
    t0("k_big_deposit");
    k_big_deposit<<<grid, kBigThreads, fixed, st>>>(a.walkers);
    t1("k_big_deposit");
  }
  if ((ph & 8) && a.any_shared) {
    t0("k_big_refresh");
    k_big_refresh<<<grid, kBigThreads, fixed, st>>>(a.walkers);
    t1("k_big_refresh");
  }
  if (ph & 16) {
    t0("k_big_force");
    k_big_force<<<dim3((a.max_atoms + kBigThreads - 1) / kBigThreads, a.nw), kBigThreads, fixed, st>>>(
        a.walkers, a.forces, a.foff, a.force_step_off, a.mode, a.step);
    t1("k_big_force");
  }
  if ((ph & 16) && a.md) {
    t0("k_big_move");
    k_big_move<<<dim3((a.max_atoms + kBigThreads - 1) / kBigThreads, a.nw), kBigThreads, 0, st>>>(
        a.walkers, *a.md, a.xio, a.coff, a.traj, a.toff, a.traj_step_off, a.step);
    t1("k_big_move");
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- hill records

// One CTA per (record, block of stencil nodes): the record's axis state from
// its centre, its tables, and a plain FP64 read-modify-write of the shadow
// (records of one launch have disjoint boxes), or the FP32 refresh.
__global__ void __launch_bounds__(kBigThreads) k_apply_hills(const WalkerDev *shape, const HillDev *recs, int refresh) {
  extern __shared__ __align__(32) unsigned char smem[];
  Grp g = big_group();
  GroupFixed<float> *fx = reinterpret_cast<GroupFixed<float> *>(smem);
  const int *src = reinterpret_cast<const int *>(shape);
  int *dst = reinterpret_cast<int *>(&fx->wd);
  for (int i = g.t; i < (int)(sizeof(WalkerDev) / 4); i += g.G) dst[i] = src[i];
  const HillDev r = recs[blockIdx.x];
  if (g.t == 0) {
    fx->clamped = 0;
    fx->flags = 0;
  }
  g.sync();
  const GridDev &gd = fx->wd.g;
  if (g.t < kMaxCv) {
    float h = (float)r.s[g.t];
    fx->sh[g.t] = h;
    fx->sl[g.t] = (float)(r.s[g.t] - (double)h);
  }
  g.sync();
  if (g.t < gd.d) axis_setup<float>(fx, g.t, true);
  g.sync();
  build_tables<float>(g, fx);
  g.sync();
  const WalkerDev &wd = fx->wd;
  const int d = gd.d;
  const int s0 = 2 * wd.R[0] + 1, s1 = d > 1 ? 2 * wd.R[1] + 1 : 1, s2 = d > 2 ? 2 * wd.R[2] + 1 : 1;
  const int total = s0 * s1 * s2;
  const int first = blockIdx.y * kStencilPerBlock, last = min(total, first + kStencilPerBlock);
  const long long n0 = gd.n[0], n01 = n0 * (d > 1 ? gd.n[1] : 1);
  const float hf = (float)r.h;
  for (int idx = first + g.t; idx < last; idx += g.G) {
    int o0 = idx % s0, rr = idx / s0, o1 = rr % s1, o2 = rr / s1;
    int j0 = fx->tabJ[0][o0];
    int j1 = d > 1 ? fx->tabJ[1][o1] : 0;
    int j2 = d > 2 ? fx->tabJ[2][o2] : 0;
    if ((j0 | j1 | j2) < 0) continue;
    const long long node = chk_node(gd, j0 + n0 * j1 + n01 * j2);
    double *p = gd.shadow + node * 4;
    if (!refresh) {
      float G = hf * fx->tabG[0][o0];
      if (d > 1) G = G * fx->tabG[1][o1];
      if (d > 2) G = G * fx->tabG[2][o2];
      p[0] += (double)G;
      p[1] += (double)__fmul_rn(G, fx->tabD[0][o0]);
      if (d > 1) p[2] += (double)__fmul_rn(G, fx->tabD[1][o1]);
      if (d > 2) p[3] += (double)__fmul_rn(G, fx->tabD[2][o2]);
    } else {
      float hi[4], lo[4];
      for (int q = 0; q < 4; ++q) {
        double v = q <= d ? p[q] : 0.0;
        hi[q] = (float)v;
        lo[q] = (float)(v - (double)hi[q]);
      }
      unsigned char *rec = reinterpret_cast<unsigned char *>(gd.rec) + node * gd.rec_bytes;
      if (d == 1) {
        *reinterpret_cast<float4 *>(rec) = make_float4(hi[0], hi[1], lo[0], lo[1]);
      } else {
        float4 *q = reinterpret_cast<float4 *>(rec);
        q[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        q[1] = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
  }
}

cudaError_t launch_apply_hills(const WalkerDev *shape, const HillDev *recs, int n, int max_stencil, bool refresh,
                               cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  dim3 grid(n, (max_stencil + kStencilPerBlock - 1) / kStencilPerBlock);
  k_apply_hills<<<grid, kBigThreads, fixed_bytes_f(), st>>>(shape, recs, refresh ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t read_hill_heads(const WalkerDev *const *wd_host, int n, double *s3h, int *dep, cudaStream_t st) {
  // wd_host[i] is a host copy of walker i's descriptor (for its jscratch)
  cudaError_t e = cudaStreamSynchronize(st);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    BigHead head;
    e = cudaMemcpy(&head, wd_host[i]->jscratch, sizeof head, cudaMemcpyDeviceToHost);
    for (int k = 0; k < 3; ++k) s3h[4 * i + k] = (double)head.sh[k] + (double)head.sl[k];
    s3h[4 * i + 3] = head.h;
    dep[i] = head.dep && !head.bad;
  }
  return e;
}

size_t big_cn_smem(const WalkerDev &hd) {
  int k = big_cn_index(hd);
  if (k < 0) return 0;
  return (size_t)hd.cv[k].na * 16 + (size_t)(kBigThreads / 32) * hd.cv[k].na * 12;
}

}  // namespace abp
