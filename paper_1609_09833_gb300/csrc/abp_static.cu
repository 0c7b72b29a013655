// abp_static.cu -- abp_step_static: the plain-form step of one walker for
// callers that cannot allocate device memory.
//
// Some callers cannot have the bias allocate device memory inside a step: a
// plugin whose host MD engine hands out GPU memory from its own fixed pool, a
// step loop that a device-wide cudaFree synchronisation would stall, a long
// run under a per-process memory limit where the bias must not fail for want
// of memory. For them this entry point runs the same three plain-form
// kernels (CV, deposit, interpolation and force) as abp_step_plain, but every
// piece of state those kernels need beyond the caller's own buffers (the
// walker's descriptor, its atom lists, the CV Jacobian scratch passed between
// the kernels, the walker state and a counter) lives in one file-scope static
// __device__ array of ABP_STATIC_SCRATCH_BYTES. The runtime reserves that
// array when it loads this module on a device and holds it until the process
// exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "abp.h"
#include "abp_internal.cuh"
#include "abp_launch.h"

using namespace abp;

namespace {

// The shared scratch. All calls (on a device) use the same bytes.
static __device__ __align__(256) unsigned char g_static_scratch[ABP_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_ptr[kMaxDevices] = {nullptr};  // device address of the array, per device

// errors are reported through abp_last_error()
abp_status sfail(abp_status code, const char *msg) { return record_error(code, msg); }

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
abp_status scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return sfail(ABP_ERR_CUDA, "abp_step_static: cudaGetSymbolAddress of the scratch array failed");
    }
    g_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_ptr[dev];
  return ABP_OK;
}

bool unique_in_range(const int32_t *idx, int n, int natoms) {
  if (n > 0 && !idx) return false;
  std::vector<int32_t> v(idx, idx + n);
  for (int32_t x : v)
    if (x < 0 || x >= natoms) return false;
  std::sort(v.begin(), v.end());
  return std::adjacent_find(v.begin(), v.end()) == v.end();
}

}  // namespace

extern "C" abp_status abp_step_static(int device, void *cuda_stream, const abp_grid_desc *gdsc, void *grid_records_dev,
                                      const abp_walker_desc *w, const void *coords_dev, int coords_dtype,
                                      void *forces_dev, int mode, int64_t step) {
  if (!gdsc || !grid_records_dev || !w || !coords_dev || !forces_dev)
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: NULL argument");
  const int d = gdsc->ncv;
  if (d < 1 || d > 3) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: ncv must be 1..3");
  if (gdsc->precision != ABP_PREC_FP32_COMP && gdsc->precision != ABP_PREC_FP64)
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: unknown precision");
  const int fp64 = gdsc->precision == ABP_PREC_FP64;
  if (coords_dtype != (fp64 ? ABP_F64 : ABP_F32))
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: coordinate dtype does not match the grid precision");
  if (mode != ABP_FORCES_ACCUMULATE && mode != ABP_FORCES_OVERWRITE)
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: bad mode");
  if (step < 0) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: step must be >= 0");
  const uintptr_t align = fp64 ? 32 : 16;
  if ((reinterpret_cast<uintptr_t>(coords_dev) | reinterpret_cast<uintptr_t>(forces_dev) |
       reinterpret_cast<uintptr_t>(grid_records_dev)) & (align - 1))
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: buffers must be 16-byte (FP64: 32-byte) aligned");
  if (w->natoms < 1) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: natoms must be >= 1");
  if (w->method != ABP_METHOD_WT) return sfail(ABP_ERR_UNSUPPORTED, "abp_step_static: well-tempered walkers only");
  if (!(w->kwall >= 0) || !std::isfinite(w->kwall))
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: kwall must be finite and >= 0");
  if (!(w->gamma > 1) || !(w->kT > 0) || w->stride < 1 || !(w->w >= 0) || !std::isfinite(w->w) || !(w->cutoff > 0))
    return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: need gamma > 1, kT > 0, w >= 0, cutoff > 0, stride >= 1");

  // grid geometry (the node convention of abp_create_grid)
  WalkerDev hd{};
  GridDev &gd = hd.g;
  gd.d = d;
  long long nodes = 1;
  for (int k = 0; k < 3; ++k) {
    bool on = k < d;
    if (on && (gdsc->n[k] < 2 || !(gdsc->hi[k] > gdsc->lo[k]) || !std::isfinite(gdsc->lo[k]) ||
               !std::isfinite(gdsc->hi[k])))
      return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: every axis needs n >= 2 and finite lo < hi");
    gd.n[k] = on ? gdsc->n[k] : 1;
    gd.periodic[k] = on ? (gdsc->periodic[k] != 0) : 0;
    gd.lo[k] = on ? gdsc->lo[k] : 0.0;
    double L = on ? gdsc->hi[k] - gdsc->lo[k] : 1.0;
    gd.D[k] = on ? (gd.periodic[k] ? L / gd.n[k] : L / (gd.n[k] - 1)) : 1.0;
    gd.invD[k] = 1.0 / gd.D[k];
    gd.L[k] = L;
    gd.u0[k] = -gd.lo[k] * gd.invD[k];
    gd.inv_n[k] = 1.0 / gd.n[k];
    gd.invD_h[k] = (float)gd.invD[k];
    gd.invD_l[k] = (float)(gd.invD[k] - (double)gd.invD_h[k]);
    gd.u0_h[k] = (float)gd.u0[k];
    gd.u0_l[k] = (float)(gd.u0[k] - (double)gd.u0_h[k]);
    if (on) nodes *= gd.n[k];
  }
  gd.prec = gdsc->precision;
  gd.rec_bytes = d == 1 ? 16 : 32;
  gd.nodes = nodes;
  gd.rec = grid_records_dev;

  // hills
  hd.natoms = w->natoms;
  hd.id = -1;
  hd.kwall = w->kwall;
  hd.kwall_f = (float)w->kwall;
  for (int k = 0; k < d; ++k) {
    if (w->kwall > 0 && !std::isfinite(w->smax[k]))
      return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: smax must be finite when kwall > 0");
    hd.smax[k] = w->kwall > 0 ? w->smax[k] : 0.0;
    hd.smax_f[k] = (float)hd.smax[k];
  }
  for (int k = 0; k < d; ++k) {
    double sig = w->sigma[k];
    if (!(sig > 0) || !std::isfinite(sig)) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: sigma must be > 0");
    double Rd = std::ceil(w->cutoff * sig / gd.D[k]);
    if (Rd > kRMax) return sfail(ABP_ERR_UNSUPPORTED, "abp_step_static: stencil half-width exceeds 64 nodes");
    hd.R[k] = (int)Rd;
    if (gd.periodic[k] && 2 * hd.R[k] + 1 > gd.n[k])
      return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: periodic stencil box wider than its axis");
    hd.sigma[k] = sig;
    hd.inv2s2[k] = 1.0 / (2.0 * sig * sig);
    hd.invs2[k] = 1.0 / (sig * sig);
  }
  hd.w = w->w;
  hd.inv_dT = 1.0 / ((w->gamma - 1.0) * w->kT);
  hd.stride = w->stride;

  // scratch layout: counters | offsets | state | descriptor | lists | Jacobian scratch
  const size_t off_ctr = 0, off_offs = 128, off_state = 256, off_wd = 512;
  size_t off = up(off_wd + sizeof(WalkerDev), 256);
  struct Piece {
    size_t off;
    std::vector<unsigned char> bytes;
  };
  std::vector<Piece> pieces;
  auto put = [&](const void *src, size_t n) -> size_t {
    size_t at = up(off, 16);
    Piece p{at, std::vector<unsigned char>(n)};
    if (n) std::memcpy(p.bytes.data(), src, n);
    pieces.push_back(std::move(p));
    off = at + n;
    return at;
  };
  size_t cv_ia[3], cv_ib[3], cv_wa[3], cv_wb[3], cv_wa64[3], cv_wb64[3];
  for (int k = 0; k < d; ++k) {
    const abp_cv_desc &c = w->cv[k];
    CvDev &cv = hd.cv[k];
    cv.type = c.type;
    cv.na = c.n_a;
    cv.nb = c.type == ABP_CV_DIHEDRAL ? 0 : c.n_b;
    if (c.type == ABP_CV_COM_DIST || c.type == ABP_CV_COORD) {
      if (c.n_a < 1 || c.n_b < 1) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: CV groups must be non-empty");
    } else if (c.type == ABP_CV_DIHEDRAL) {
      if (c.n_a != 4) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: a dihedral needs 4 atoms");
    } else if (c.type == ABP_CV_RMSD) {
      return sfail(ABP_ERR_UNSUPPORTED, "abp_step_static: RMSD CVs are not built for this entry point");
    } else {
      return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: unknown CV type");
    }
    if (c.type == ABP_CV_COORD) {
      if (c.nn != 6 || c.mm != 12)
        return sfail(ABP_ERR_UNSUPPORTED, "abp_step_static: only the n = 6, m = 12 switching function is built");
      if (!(c.r0 > 0)) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: r0 must be > 0");
      cv.inv_r0sq = 1.0 / (c.r0 * c.r0);
    }
    if (!unique_in_range(c.idx_a, cv.na, w->natoms) || !unique_in_range(c.idx_b, cv.nb, w->natoms))
      return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: atom index lists must be unique and in [0, natoms)");
    cv.pbc = c.pbc != 0;
    cv.hp = !fp64 && c.type == ABP_CV_DIHEDRAL && hd.sigma[k] < kDihedralHpWidth;
    for (int q = 0; q < 3; ++q) {
      if (cv.pbc && !(c.box[q] > 0)) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: pbc needs box edges > 0");
      cv.box[q] = cv.pbc ? c.box[q] : 0.0;
      cv.inv_box[q] = cv.pbc ? 1.0 / c.box[q] : 0.0;
    }
    cv_ia[k] = put(c.idx_a, sizeof(int32_t) * cv.na);
    cv_ib[k] = put(cv.nb ? c.idx_b : nullptr, sizeof(int32_t) * cv.nb);
    cv_wa[k] = cv_wb[k] = cv_wa64[k] = cv_wb64[k] = 0;
    if (c.type == ABP_CV_COM_DIST) {
      for (int grp = 0; grp < 2; ++grp) {
        int n = grp ? cv.nb : cv.na;
        const double *m = grp ? c.mass_b : c.mass_a;
        std::vector<double> wd(n);
        std::vector<float> wf(n);
        double M = 0;
        for (int i = 0; i < n; ++i) {
          double mi = m ? m[i] : 1.0;
          if (!(mi > 0) || !std::isfinite(mi)) return sfail(ABP_ERR_INVALID_ARG, "abp_step_static: masses must be > 0");
          wd[i] = mi;
          M += mi;
        }
        bool equal = true;
        for (int i = 0; i < n; ++i) {
          wd[i] /= M;
          wf[i] = (float)wd[i];
          equal = equal && wd[i] == wd[0];
        }
        (grp ? cv.wc_b : cv.wc_a) = equal ? (float)(wd[0] / (double)wf[0] - 1.0) : 0.f;
        (grp ? cv_wb[k] : cv_wa[k]) = put(wf.data(), sizeof(float) * n);
        (grp ? cv_wb64[k] : cv_wa64[k]) = put(wd.data(), sizeof(double) * n);
      }
    }
  }
  const size_t off_js = up(off, 256);
  const size_t total = off_js + (size_t)plain_scratch_bytes(fp64, hd.cv, d);
  if (total > ABP_STATIC_SCRATCH_BYTES)
    return sfail(ABP_ERR_INVALID_ARG,
                 "abp_step_static: this walker needs more static scratch than ABP_STATIC_SCRATCH_BYTES (1 MiB)");
  const int threads = 128;
  const int dyn = group_layout(hd.natoms, hd.cv, gd, hd.R, threads / 32, fp64 ? 32 : 16, 0).total;
  if (group_fixed_bytes(fp64) + dyn > 227 * 1024)
    return sfail(ABP_ERR_UNSUPPORTED, "abp_step_static: the walker needs more shared memory than an SM has");

  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(ABP_ERR_CUDA, "abp_step_static: cudaSetDevice failed");
  }
  struct Restore {
    int dev;
    ~Restore() {
      if (dev >= 0) cudaSetDevice(dev);
    }
  } restore{prev_dev};
  unsigned char *base = nullptr;
  abp_status st = scratch_address(device, &base);
  if (st) return st;

  // device addresses inside the scratch
  for (int k = 0; k < d; ++k) {
    CvDev &cv = hd.cv[k];
    cv.ia = reinterpret_cast<const int32_t *>(base + cv_ia[k]);
    cv.ib = reinterpret_cast<const int32_t *>(base + cv_ib[k]);
    if (cv.type == ABP_CV_COM_DIST) {
      cv.wa = reinterpret_cast<const float *>(base + cv_wa[k]);
      cv.wb = reinterpret_cast<const float *>(base + cv_wb[k]);
      cv.wa64 = reinterpret_cast<const double *>(base + cv_wa64[k]);
      cv.wb64 = reinterpret_cast<const double *>(base + cv_wb64[k]);
    }
  }
  hd.fbuf = nullptr;
  hd.jscratch = base + off_js;
  hd.state = reinterpret_cast<WalkerState *>(base + off_state);

  // one staging image of everything the kernels read, copied in one call;
  // the counters start at zero on every call
  std::vector<unsigned char> img(off_js, 0);
  const long long zero_offs[2] = {0, 0};
  std::memcpy(img.data() + off_offs, zero_offs, sizeof zero_offs);
  std::memcpy(img.data() + off_wd, &hd, sizeof hd);
  for (const Piece &p : pieces)
    if (!p.bytes.empty()) std::memcpy(img.data() + p.off, p.bytes.data(), p.bytes.size());
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  e = cudaMemcpyAsync(base, img.data(), img.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(ABP_ERR_CUDA, "abp_step_static: copy of the walker image into the scratch failed");
  }

  const WalkerDev *wd_dev = reinterpret_cast<const WalkerDev *>(base + off_wd);
  const long long *offs = reinterpret_cast<const long long *>(base + off_offs);
  int dep = (step % w->stride) == 0;
  PlainArgs a{};
  a.nw = 1;
  a.wd_dev = &wd_dev;
  a.dyn_bytes = &dyn;
  a.deposit = &dep;
  a.threads = threads;
  a.coords = coords_dev;
  a.coff = offs;
  a.forces = forces_dev;
  a.foff = offs;
  a.mode = mode;
  a.step = step;
  a.log = DepositLog{nullptr, nullptr, 0};
  a.ctr = reinterpret_cast<DevCounters *>(base + off_ctr);
  e = launch_plain(a, fp64, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(ABP_ERR_CUDA, "abp_step_static: kernel launch failed");
  }
  return ABP_OK;
}
