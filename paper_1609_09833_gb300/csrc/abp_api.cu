// abp_api.cu -- host implementation of the C ABI declared in include/abp.h.
// Owns every device allocation (grids, walker descriptors, force buffers,
// deposit log), validates arguments, and launches the kernels of
// abp_kernels.cu on the context stream. No exception leaves this file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "abp.h"
#include "abp_internal.cuh"
#include "abp_launch.h"

using namespace abp;

namespace {

thread_local std::string g_err;

abp_status fail(abp_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(ABP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Per-kernel timing of a context: an event pair per launch, accumulated per
// kernel name when read (abp_kernel_times).
struct KernelTimer final : LaunchTimer {
  struct Pending {
    std::string name;
    cudaEvent_t a, b;
    bool open;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<std::string, std::pair<long long, double>>> totals;
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
    }
    return e;
  }
  void begin(const char *kernel, cudaStream_t st) override {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cudaEvent_t a = take(), b = take();
    if (!a || !b) {
      if (a) pool.push_back(a);
      if (b) pool.push_back(b);
      return;
    }
    cudaEventRecord(a, st);
    pending.push_back(Pending{kernel, a, b, true});
  }
  void end(const char *kernel, cudaStream_t st) override {
    if (!pending.empty() && pending.back().open && pending.back().name == kernel) {
      cudaEventRecord(pending.back().b, st);
      pending.back().open = false;
    }
  }
  // accumulate the finished pairs (caller has synchronised)
  void collect() {
    for (auto &p : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        auto it = std::find_if(totals.begin(), totals.end(), [&](const auto &t) { return t.first == p.name; });
        if (it == totals.end()) {
          totals.push_back({p.name, {0, 0.0}});
          it = totals.end() - 1;
        }
        it->second.first += 1;
        it->second.second += ms;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  ~KernelTimer() override {
    for (auto &p : pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct TableCache {
  std::vector<TableEntry> key;
  TableEntry *dev = nullptr;
  size_t cap = 0;
  unsigned long long last_use = 0;
};

}  // namespace

namespace abp {
abp_status record_error(abp_status code, const char *msg) { return fail(code, "%s", msg); }

cudaError_t smem_attr(const void *fn, size_t bytes) {
  struct Given {
    const void *fn;
    int dev;
    size_t bytes;
  };
  static std::mutex mu;
  static std::vector<Given> given;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  for (Given &g : given)
    if (g.fn == fn && g.dev == dev) {
      if (g.bytes >= bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) g.bytes = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) given.push_back(Given{fn, dev, bytes});
  return e;
}
}  // namespace abp

struct abp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t used = 0;
  DevCounters *ctr = nullptr;
  DepositLog log{nullptr, nullptr, 0};
  TableCache tables[6];
  unsigned long long use_clock = 0;
  int next_id = 0;
  int sms = 0;  // multiprocessors of the device
  int tune_G = 0, tune_gpc = 0, tune_tile = -1;  // tile -1: library default (off; opt in with 1)
  int tune_lean = 0;
  std::vector<BigItem> big_key;                   // phased-form item lists of the last call
  BigItem *big_dev = nullptr;
  size_t big_cap = 0;
  HillDev *hill_dev = nullptr;  // hill records of the last abp_grid_apply_hills
  size_t hill_cap = 0;
  KernelTimer *timer = nullptr;  // ABP_TUNE_TIMING
  std::mutex mu;
};

struct abp_grid {
  abp_ctx *ctx = nullptr;
  GridDev g{};
  abp_grid_desc desc{};
  size_t bytes = 0;
  size_t shadow_bytes = 0;
};

struct abp_walker {
  abp_ctx *ctx = nullptr;
  abp_grid *grid = nullptr;
  WalkerDev hd{};
  WalkerDev *dd = nullptr;
  std::vector<std::pair<void *, size_t>> allocs;
  bool has_cn = false;
  bool big = false;    // runs in the phased form (shared grid, or too large for a walker group)
  bool win = false;    // runs in the windowed form of the fused kernel (COM distance / dihedral CVs)
  bool has_rmsd = false;
  // the closed-loop kernel's register-fed form applies: FP32 WT walkers of at
  // most 64 atoms of at most two a5 terms each, COM groups of at most 16
  // atoms, the other CVs dihedrals
  bool md_fast = false;
  long long cost = 0;  // rough work estimate used to order batched launches
};

namespace {

abp_status set_device(const abp_ctx *ctx) {
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur));
  if (cur != ctx->device) CUDA_TRY(cudaSetDevice(ctx->device));
  return ABP_OK;
}

abp_status dev_alloc(abp_ctx *ctx, size_t bytes, void **out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->used + bytes > ctx->budget)
    return fail(ABP_ERR_ADMISSION, "allocation of %zu bytes exceeds the HBM budget (%zu of %zu used)", bytes,
                ctx->used, ctx->budget);
  cudaError_t e = cudaMalloc(out, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return fail(ABP_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->used += bytes;
  return ABP_OK;
}

void dev_free(abp_ctx *ctx, void *p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  if (bytes == 0) bytes = 16;
  ctx->used -= std::min(ctx->used, bytes);
}

int rec_bytes(int prec, int d) {
  (void)prec;
  return d == 1 ? 16 : 32;
}

double spacing(const abp_grid_desc &d, int k) {
  return d.periodic[k] ? (d.hi[k] - d.lo[k]) / d.n[k] : (d.hi[k] - d.lo[k]) / (d.n[k] - 1);
}

int walker_fp64(const abp_walker *w) { return w->grid->desc.precision == ABP_PREC_FP64; }

// Dynamic shared bytes of one walker group without a tile.
int dyn_bytes(const abp_walker *w, int nwarps) {
  return group_layout(w->hd.natoms, w->hd.cv, w->hd.g, w->hd.R, nwarps, walker_fp64(w) ? 32 : 16, 0).total;
}

// Common validation of a walker list. Returns the precision (0/1) via *fp64.
abp_status check_list(abp_ctx *ctx, abp_walker *const *walkers, int n, int *fp64, bool *shared) {
  if (n < 0) return fail(ABP_ERR_INVALID_ARG, "negative walker count");
  if (n > 0 && !walkers) return fail(ABP_ERR_INVALID_ARG, "walker list is NULL");
  int prec = -1;
  thread_local std::vector<const abp_grid *> grids;  // reused: no allocation per call
  grids.clear();
  *shared = false;
  for (int i = 0; i < n; ++i) {
    const abp_walker *w = walkers[i];
    if (!w) return fail(ABP_ERR_INVALID_ARG, "walker %d is NULL", i);
    if (w->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "walker %d belongs to another context", i);
    int p = walker_fp64(w);
    if (prec >= 0 && p != prec) return fail(ABP_ERR_INVALID_ARG, "walkers of one call must share a grid precision");
    prec = p;
    grids.push_back(w->grid);
  }
  std::sort(grids.begin(), grids.end());
  *shared = std::adjacent_find(grids.begin(), grids.end()) != grids.end();
  *fp64 = prec < 0 ? 0 : prec;
  return ABP_OK;
}

// Device table for a walker list (cached: a small LRU of recent lists).
abp_status get_table(abp_ctx *ctx, abp_walker *const *walkers, int n, bool sort_by_cost, const TableEntry **out) {
  std::vector<TableEntry> key(n);
  for (int i = 0; i < n; ++i) key[i] = TableEntry{walkers[i]->dd, i, 0};
  if (sort_by_cost) {
    std::vector<long long> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = walkers[i]->cost;
    std::stable_sort(key.begin(), key.end(),
                     [&](const TableEntry &a, const TableEntry &b) { return cost[a.idx] > cost[b.idx]; });
  }
  ++ctx->use_clock;
  TableCache *victim = &ctx->tables[0];
  for (auto &t : ctx->tables) {
    if (t.dev && t.key.size() == key.size() &&
        std::memcmp(t.key.data(), key.data(), key.size() * sizeof(TableEntry)) == 0) {
      t.last_use = ctx->use_clock;
      *out = t.dev;
      return ABP_OK;
    }
    if (t.last_use < victim->last_use) victim = &t;
  }
  size_t need = std::max<size_t>(1, key.size()) * sizeof(TableEntry);
  if (victim->cap < need) {
    if (victim->dev) cudaFree(victim->dev);
    victim->dev = nullptr;
    victim->cap = 0;
    CUDA_TRY(cudaMalloc(&victim->dev, need));
    victim->cap = need;
  }
  // pageable source: the runtime stages it before returning, so `key` may die
  CUDA_TRY(cudaMemcpyAsync(victim->dev, key.data(), key.size() * sizeof(TableEntry), cudaMemcpyHostToDevice,
                           ctx->stream));
  victim->key = std::move(key);
  victim->last_use = ctx->use_clock;
  *out = victim->dev;
  return ABP_OK;
}

// Launch shape for a batch: a group of G threads per walker, several
// groups per CTA, as shared memory allows. Multi-step launches of FP32
// walkers with few enough walkers per SM also give each group a shared-memory
// tile of its grid (the rest of ~220 KB / walkers-per-SM). A windowed batch
// defaults to one 256-thread group per CTA: its two halves run the window
// pipeline's two stages.
// The per-step form's shape from the batch's largest group footprint gb
// (bytes at g threads per group, with tile budget tb): groups per CTA as
// shared memory allows.
abp_status step_shape(const abp_ctx *ctx, bool cn, int g, int gb, int tb, int *G, int *gpc, int *group_bytes,
                      int *tile_budget) {
  const int smem_max = 227 * 1024;
  if (gb > smem_max) return fail(ABP_ERR_UNSUPPORTED, "a walker needs %d bytes of shared memory (max %d)", gb, smem_max);
  int per = 1;
  if (tb == 0) per = ctx->tune_gpc ? ctx->tune_gpc : (cn ? 2 : 4);
  while (per > 1 && (per * gb > (ctx->tune_gpc ? smem_max : 100 * 1024) || per * g > 256)) --per;
  *G = g;
  *gpc = per;
  *group_bytes = gb;
  *tile_budget = tb;
  return ABP_OK;
}

abp_status pick_shape(const abp_ctx *ctx, abp_walker *const *walkers, int n, int fp64, int nsteps, bool window,
                      int *G, int *gpc, int *group_bytes, int *tile_budget) {
  bool cn = false;
  for (int i = 0; i < n; ++i) cn = cn || walkers[i]->has_cn;
  if (window) {
    const int g = ctx->tune_G ? ctx->tune_G : 256;
    int gb = 0;
    for (int i = 0; i < n; ++i) gb = std::max(gb, run_group_bytes(walkers[i]->hd, fp64, g, 0, true));
    const int smem_max = 227 * 1024;
    if (gb > smem_max) return fail(ABP_ERR_UNSUPPORTED, "a walker needs %d bytes of shared memory (max %d)", gb, smem_max);
    int per = ctx->tune_gpc ? ctx->tune_gpc : 1;
    while (per > 1 && (per * gb > smem_max || per * g > 256)) --per;
    *G = g;
    *gpc = per;
    *group_bytes = gb;
    *tile_budget = 0;
    return ABP_OK;
  }
  const int g = ctx->tune_G ? ctx->tune_G : (cn ? 128 : 32);
  int fixed = group_fixed_bytes(fp64);
  int tb = 0;
  // Measured on the 64-walker workload, one warp per walker: reloading and
  // indexing the tile cost more than the L2 reads it saves, so tiles are
  // opt-in (ABP_TUNE_TILE = 1) and need a multi-step launch.
  bool tile_ok = ctx->tune_tile == 1 && nsteps >= 8;
  if (!fp64 && tile_ok && ctx->sms > 0) {
    int per_sm = (n + ctx->sms - 1) / ctx->sms;
    int avail = (220 * 1024) / per_sm - fixed - 1024;
    if (avail > 16 * 1024) tb = avail;
  }
  int gb = 0;
  bool any_tile = false;
  for (int i = 0; i < n; ++i) {
    int b = run_group_bytes(walkers[i]->hd, fp64, g, tb, false);
    gb = std::max(gb, b);
    if (tb > 0 && b > run_group_bytes(walkers[i]->hd, fp64, g, 0, false)) any_tile = true;
  }
  if (tb > 0 && !any_tile) {
    tb = 0;
    gb = 0;
    for (int i = 0; i < n; ++i) gb = std::max(gb, run_group_bytes(walkers[i]->hd, fp64, g, 0, false));
  }
  return step_shape(ctx, cn, g, gb, tb, G, gpc, group_bytes, tile_budget);
}

}  // namespace

extern "C" {

const char *abp_last_error(void) { return g_err.c_str(); }
const char *abp_version(void) { return "abp-gb300 0.1 (sm_103a)"; }

abp_status abp_ctx_create(abp_ctx **out, int device, void *cuda_stream, size_t hbm_budget_bytes) {
  if (!out) return fail(ABP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(ABP_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, ndev);
  abp_ctx *c = new (std::nothrow) abp_ctx();
  if (!c) return fail(ABP_ERR_OOM, "host allocation failed");
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->budget = hbm_budget_bytes;
  abp_status st = set_device(c);
  if (st == ABP_OK && cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) c->sms = 0;
  if (st == ABP_OK) {
    cudaError_t e = cudaMalloc(&c->ctr, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMemset(c->ctr, 0, sizeof(DevCounters));
    if (e != cudaSuccess) st = fail(ABP_ERR_CUDA, "counter allocation: %s", cudaGetErrorString(e));
  }
  if (st != ABP_OK) {
    if (c->ctr) cudaFree(c->ctr);
    delete c;
    return st;
  }
  *out = c;
  return ABP_OK;
}

abp_status abp_ctx_set_stream(abp_ctx *ctx, void *cuda_stream) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return ABP_OK;
}

abp_status abp_ctx_tune(abp_ctx *ctx, int knob, int value) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  switch (knob) {
    case ABP_TUNE_GROUP_THREADS:
      if (value != 0 && value != 32 && value != 64 && value != 128 && value != 256)
        return fail(ABP_ERR_INVALID_ARG, "group threads must be 32, 64, 128 or 256");
      ctx->tune_G = value;
      return ABP_OK;
    case ABP_TUNE_GROUPS_PER_CTA:
      if (value < 0 || value > kMaxGroupsPerCta) return fail(ABP_ERR_INVALID_ARG, "groups per CTA must be 0..8");
      ctx->tune_gpc = value;
      return ABP_OK;
    case ABP_TUNE_TILE:
      if (value < -1 || value > 1) return fail(ABP_ERR_INVALID_ARG, "tile knob must be -1, 0 or 1");
      ctx->tune_tile = value;
      return ABP_OK;
    case ABP_TUNE_LEAN:
      if (value < 0 || value > 1) return fail(ABP_ERR_INVALID_ARG, "lean knob must be 0 or 1");
      ctx->tune_lean = value;
      return ABP_OK;
    case ABP_TUNE_TIMING:
      if (value < 0 || value > 1) return fail(ABP_ERR_INVALID_ARG, "timing knob must be 0 or 1");
      if (value && !ctx->timer) ctx->timer = new (std::nothrow) KernelTimer();
      if (value && !ctx->timer) return fail(ABP_ERR_OOM, "timer");
      if (!value && ctx->timer) {
        cudaStreamSynchronize(ctx->stream);
        delete ctx->timer;
        ctx->timer = nullptr;
      }
      return ABP_OK;
  }
  return fail(ABP_ERR_INVALID_ARG, "unknown knob %d", knob);
}

abp_status abp_ctx_bytes(const abp_ctx *ctx, size_t *used, size_t *budget) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  if (used) *used = ctx->used;
  if (budget) *budget = ctx->budget;
  return ABP_OK;
}

void abp_ctx_destroy(abp_ctx *ctx) {
  if (!ctx) return;
  set_device(ctx);
  cudaStreamSynchronize(ctx->stream);
  for (auto &t : ctx->tables)
    if (t.dev) cudaFree(t.dev);
  if (ctx->big_dev) cudaFree(ctx->big_dev);
  if (ctx->hill_dev) cudaFree(ctx->hill_dev);
  if (ctx->log.rec) cudaFree(ctx->log.rec);
  if (ctx->log.count) cudaFree(ctx->log.count);
  if (ctx->ctr) cudaFree(ctx->ctr);
  delete ctx->timer;
  delete ctx;
}

abp_status abp_kernel_times(abp_ctx *ctx, abp_kernel_time *out, int cap, int *n_out) {
  if (!ctx || !n_out || (cap > 0 && !out)) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  *n_out = 0;
  if (!ctx->timer) return ABP_OK;
  abp_status st = set_device(ctx);
  if (st) return st;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->timer->collect();
  int n = 0;
  for (const auto &t : ctx->timer->totals) {
    if (n >= cap) break;
    std::memset(&out[n], 0, sizeof(abp_kernel_time));
    std::snprintf(out[n].name, sizeof out[n].name, "%s", t.first.c_str());
    out[n].launches = t.second.first;
    out[n].ms = t.second.second;
    ++n;
  }
  ctx->timer->totals.clear();
  *n_out = n;
  return ABP_OK;
}

// ---------------------------------------------------------------- grids

abp_status abp_create_grid(abp_ctx *ctx, const abp_grid_desc *d, abp_grid **out) {
  if (!ctx || !d || !out) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (d->ncv < 1 || d->ncv > 3) return fail(ABP_ERR_INVALID_ARG, "ncv must be 1..3 (got %d)", d->ncv);
  if (d->precision != ABP_PREC_FP32_COMP && d->precision != ABP_PREC_FP64)
    return fail(ABP_ERR_INVALID_ARG, "unknown precision %d", d->precision);
  if (d->shared && d->precision != ABP_PREC_FP32_COMP)
    return fail(ABP_ERR_UNSUPPORTED, "shared grids are FP32_COMP grids (their accumulator is FP64)");
  long long nodes = 1;
  for (int k = 0; k < d->ncv; ++k) {
    if (d->n[k] < 2) return fail(ABP_ERR_INVALID_ARG, "axis %d needs >= 2 grid points", k);
    if (!(d->hi[k] > d->lo[k]) || !std::isfinite(d->lo[k]) || !std::isfinite(d->hi[k]))
      return fail(ABP_ERR_INVALID_ARG, "axis %d needs finite lo < hi", k);
    nodes *= d->n[k];
    if (nodes > (1ll << 34)) return fail(ABP_ERR_INVALID_ARG, "grid too large");
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  abp_status st = set_device(ctx);
  if (st) return st;
  abp_grid *g = new (std::nothrow) abp_grid();
  if (!g) return fail(ABP_ERR_OOM, "host allocation failed");
  g->ctx = ctx;
  g->desc = *d;
  GridDev &gd = g->g;
  gd.d = d->ncv;
  for (int k = 0; k < 3; ++k) {
    bool on = k < d->ncv;
    gd.n[k] = on ? d->n[k] : 1;
    gd.periodic[k] = on ? (d->periodic[k] != 0) : 0;
    gd.lo[k] = on ? d->lo[k] : 0.0;
    gd.D[k] = on ? spacing(*d, k) : 1.0;
    gd.invD[k] = 1.0 / gd.D[k];
    gd.L[k] = on ? d->hi[k] - d->lo[k] : 1.0;
    gd.u0[k] = -gd.lo[k] * gd.invD[k];
    gd.inv_n[k] = 1.0 / gd.n[k];
    gd.invD_h[k] = (float)gd.invD[k];
    gd.invD_l[k] = (float)(gd.invD[k] - (double)gd.invD_h[k]);
    gd.u0_h[k] = (float)gd.u0[k];
    gd.u0_l[k] = (float)(gd.u0[k] - (double)gd.u0_h[k]);
  }
  gd.prec = d->precision;
  gd.rec_bytes = rec_bytes(d->precision, d->ncv);
  gd.nodes = nodes;
  g->bytes = (size_t)nodes * gd.rec_bytes;
  st = dev_alloc(ctx, g->bytes, &gd.rec);
  if (st) {
    delete g;
    return st;
  }
  gd.shared = d->shared ? 1 : 0;
  gd.shadow = nullptr;
  gd.oob = &ctx->ctr->oob;  // device address of the context's counter
  if (gd.shared) {
    g->shadow_bytes = (size_t)nodes * 4 * sizeof(double);
    void *p = nullptr;
    st = dev_alloc(ctx, g->shadow_bytes, &p);
    if (st) {
      dev_free(ctx, gd.rec, g->bytes);
      delete g;
      return st;
    }
    gd.shadow = static_cast<double *>(p);
  }
  cudaError_t e = cudaMemsetAsync(gd.rec, 0, g->bytes, ctx->stream);
  if (e == cudaSuccess && gd.shadow) e = cudaMemsetAsync(gd.shadow, 0, g->shadow_bytes, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    dev_free(ctx, gd.rec, g->bytes);
    if (gd.shadow) dev_free(ctx, gd.shadow, g->shadow_bytes);
    delete g;
    return fail(ABP_ERR_CUDA, "grid clear: %s", cudaGetErrorString(e));
  }
  *out = g;
  return ABP_OK;
}

void abp_grid_destroy(abp_grid *g) {
  if (!g) return;
  std::lock_guard<std::mutex> lk(g->ctx->mu);
  set_device(g->ctx);
  cudaStreamSynchronize(g->ctx->stream);
  dev_free(g->ctx, g->g.rec, g->bytes);
  if (g->g.shadow) dev_free(g->ctx, g->g.shadow, g->shadow_bytes);
  delete g;
}

abp_status abp_grid_clear(abp_ctx *ctx, abp_grid *g) {
  if (!ctx || !g || g->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "bad grid");
  abp_status st = set_device(ctx);
  if (st) return st;
  CUDA_TRY(cudaMemsetAsync(g->g.rec, 0, g->bytes, ctx->stream));
  if (g->g.shadow) CUDA_TRY(cudaMemsetAsync(g->g.shadow, 0, g->shadow_bytes, ctx->stream));
  return ABP_OK;
}

// ---------------------------------------------------------------- walkers

namespace {

abp_status walker_alloc(abp_walker *w, size_t bytes, void **p) {
  abp_status st = dev_alloc(w->ctx, bytes, p);
  if (st == ABP_OK) w->allocs.push_back({*p, bytes});
  return st;
}

abp_status upload(abp_walker *w, const void *src, size_t bytes, void **dst) {
  abp_status st = walker_alloc(w, bytes, dst);
  if (st) return st;
  if (bytes) CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return ABP_OK;
}

void walker_free(abp_walker *w) {
  for (auto &a : w->allocs) dev_free(w->ctx, a.first, a.second);
  w->allocs.clear();
}

abp_status check_indices(const int32_t *idx, int n, int natoms, const char *what, int k) {
  if (n > 0 && !idx) return fail(ABP_ERR_INVALID_ARG, "CV %d: %s index list is NULL", k, what);
  std::vector<int32_t> v(idx, idx + n);
  for (int i = 0; i < n; ++i)
    if (v[i] < 0 || v[i] >= natoms)
      return fail(ABP_ERR_INVALID_ARG, "CV %d: %s index %d out of range [0, %d)", k, what, v[i], natoms);
  std::sort(v.begin(), v.end());
  if (std::adjacent_find(v.begin(), v.end()) != v.end())
    return fail(ABP_ERR_INVALID_ARG, "CV %d: %s index list has duplicates", k, what);
  return ABP_OK;
}

// COM weights m_i / M of group grp (0: list A, 1: list B) in FP64 (unit
// masses when none are given); false on a mass that is not finite and > 0.
bool com_weights(const abp_cv_desc &c, int grp, std::vector<double> &wd) {
  const int n = grp ? c.n_b : c.n_a;
  const double *m = grp ? c.mass_b : c.mass_a;
  wd.assign(n, 0.0);
  double M = 0;
  for (int i = 0; i < n; ++i) {
    const double mi = m ? m[i] : 1.0;
    if (!(mi > 0) || !std::isfinite(mi)) return false;
    wd[i] = mi;
    M += mi;
  }
  for (int i = 0; i < n; ++i) wd[i] = wd[i] / M;
  return true;
}

// The closed-loop form's a5 term tables, in the order the kernels' own
// build forms them: per atom its list entries CV by CV, list A before list
// B; a COM entry carries the weight as the kernels hold it (FP32 walkers:
// the FP32 weight; list B negated) on the unit separation (offset 12 k), a
// dihedral or RMSD entry -1 on its atom's gradient row (offset 12 k + 3 i).
extern "C++" {
template <typename Real>
void atom_term_tables(const abp_walker_desc *d, int ncv, std::vector<int> &cnt, std::vector<AtomTerm<Real>> &terms) {
  cnt.assign(d->natoms, 0);
  terms.assign((size_t)d->natoms * kAtomTerms, AtomTerm<Real>{(Real)0, 0});
  for (int k = 0; k < ncv; ++k) {
    const abp_cv_desc &c = d->cv[k];
    const bool com = c.type == ABP_CV_COM_DIST;
    for (int l = 0; l < (com ? 2 : 1); ++l) {
      const int n = l ? c.n_b : (c.type == ABP_CV_DIHEDRAL ? 4 : c.n_a);
      const int32_t *list = l ? c.idx_b : c.idx_a;
      std::vector<double> wd;
      if (com) com_weights(c, l, wd);
      for (int i = 0; i < n; ++i) {
        const int at = list[i];
        Real wt = (Real)-1;
        if (com) {
          wt = sizeof(Real) == 4 ? (Real)(float)wd[i] : (Real)wd[i];
          if (l) wt = -wt;
        }
        terms[(size_t)at * kAtomTerms + cnt[at]] = AtomTerm<Real>{wt, k * 12 + (com ? 0 : 3 * i)};
        cnt[at] += 1;
      }
    }
  }
}
}  // extern "C++"

abp_status build_cv(abp_walker *w, const abp_cv_desc &c, int k, int natoms, CvDev *out) {
  CvDev cv{};
  cv.type = c.type;
  cv.na = c.n_a;
  cv.nb = c.n_b;
  abp_status st;
  switch (c.type) {
    case ABP_CV_COM_DIST:
      if (c.n_a < 1 || c.n_b < 1) return fail(ABP_ERR_INVALID_ARG, "CV %d: COM groups must be non-empty", k);
      break;
    case ABP_CV_DIHEDRAL:
      if (c.n_a != 4) return fail(ABP_ERR_INVALID_ARG, "CV %d: a dihedral needs 4 atoms", k);
      cv.nb = 0;
      break;
    case ABP_CV_RMSD:
      if (c.n_a < 1 || c.n_a > 4) return fail(ABP_ERR_UNSUPPORTED, "CV %d: RMSDs of 1 to 4 atoms are supported", k);
      if (!c.ref) return fail(ABP_ERR_INVALID_ARG, "CV %d: an RMSD needs reference positions", k);
      for (int i = 0; i < 3 * c.n_a; ++i)
        if (!std::isfinite(c.ref[i])) return fail(ABP_ERR_INVALID_ARG, "CV %d: reference positions must be finite", k);
      cv.nb = 0;
      break;
    case ABP_CV_COORD:
      if (c.n_a < 1 || c.n_b < 1) return fail(ABP_ERR_INVALID_ARG, "CV %d: CN groups must be non-empty", k);
      if (c.nn != 6 || c.mm != 12)
        return fail(ABP_ERR_UNSUPPORTED, "CV %d: only the n = 6, m = 12 switching function is built", k);
      if (!(c.r0 > 0) || !std::isfinite(c.r0)) return fail(ABP_ERR_INVALID_ARG, "CV %d: r0 must be > 0", k);
      cv.inv_r0sq = 1.0 / (c.r0 * c.r0);
      break;
    default:
      return fail(ABP_ERR_INVALID_ARG, "CV %d: unknown type %d", k, c.type);
  }
  if ((st = check_indices(c.idx_a, cv.na, natoms, "A", k))) return st;
  if ((st = check_indices(c.idx_b, cv.nb, natoms, "B", k))) return st;
  cv.pbc = c.pbc != 0;
  for (int q = 0; q < 3; ++q) {
    if (cv.pbc && !(c.box[q] > 0)) return fail(ABP_ERR_INVALID_ARG, "CV %d: pbc needs box edges > 0", k);
    cv.box[q] = cv.pbc ? c.box[q] : 0.0;
    cv.inv_box[q] = cv.pbc ? 1.0 / c.box[q] : 0.0;
  }
  void *p;
  if ((st = upload(w, c.idx_a, sizeof(int32_t) * cv.na, &p))) return st;
  cv.ia = static_cast<const int32_t *>(p);
  if ((st = upload(w, cv.nb ? c.idx_b : nullptr, sizeof(int32_t) * cv.nb, &p))) return st;
  cv.ib = static_cast<const int32_t *>(p);
  if (c.type == ABP_CV_RMSD) {
    std::vector<float> rf(3 * cv.na);
    for (int i = 0; i < 3 * cv.na; ++i) rf[i] = (float)c.ref[i];
    if ((st = upload(w, rf.data(), sizeof(float) * rf.size(), &p))) return st;
    cv.ref = static_cast<const float *>(p);
    if ((st = upload(w, c.ref, sizeof(double) * 3 * cv.na, &p))) return st;
    cv.ref64 = static_cast<const double *>(p);
  }
  if (c.type == ABP_CV_COM_DIST) {
    // weights m_i / M_group, computed once in FP64
    for (int grp = 0; grp < 2; ++grp) {
      int n = grp ? cv.nb : cv.na;
      std::vector<double> wd;
      if (!com_weights(c, grp, wd)) return fail(ABP_ERR_INVALID_ARG, "CV %d: masses must be > 0", k);
      std::vector<float> wf(n);
      bool equal = true;
      for (int i = 0; i < n; ++i) {
        wf[i] = (float)wd[i];
        equal = equal && wd[i] == wd[0];
      }
      (grp ? cv.wc_b : cv.wc_a) = equal ? (float)(wd[0] / (double)wf[0] - 1.0) : 0.f;
      if ((st = upload(w, wf.data(), sizeof(float) * n, &p))) return st;
      (grp ? cv.wb : cv.wa) = static_cast<const float *>(p);
      if ((st = upload(w, wd.data(), sizeof(double) * n, &p))) return st;
      (grp ? cv.wb64 : cv.wa64) = static_cast<const double *>(p);
    }
  }
  *out = cv;
  return ABP_OK;
}

}  // namespace

abp_status abp_walker_create(abp_ctx *ctx, abp_grid *grid, const abp_walker_desc *d, abp_walker **out) {
  if (!ctx || !grid || !d || !out) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (grid->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "grid belongs to another context");
  if (d->natoms < 1) return fail(ABP_ERR_INVALID_ARG, "natoms must be >= 1");
  if (d->method == ABP_METHOD_WT &&
      (!(d->gamma > 1) || !(d->kT > 0) || d->stride < 1 || !(d->w >= 0) || !std::isfinite(d->w) ||
       !std::isfinite(d->gamma) || !std::isfinite(d->kT) || !(d->cutoff > 0)))
    return fail(ABP_ERR_INVALID_ARG, "need gamma > 1, kT > 0, w >= 0, cutoff > 0, stride >= 1");
  if (d->stride < 1) return fail(ABP_ERR_INVALID_ARG, "stride must be >= 1");
  std::lock_guard<std::mutex> lk(ctx->mu);
  abp_status st = set_device(ctx);
  if (st) return st;
  abp_walker *w = new (std::nothrow) abp_walker();
  if (!w) return fail(ABP_ERR_OOM, "host allocation failed");
  w->ctx = ctx;
  w->grid = grid;
  WalkerDev &hd = w->hd;
  hd.g = grid->g;
  hd.natoms = d->natoms;
  const int ncv = grid->desc.ncv;
  const int fp64 = grid->desc.precision == ABP_PREC_FP64;
  const bool mabp = d->method == ABP_METHOD_MABP;
  if (d->method != ABP_METHOD_WT && !mabp) {
    delete w;
    return fail(ABP_ERR_INVALID_ARG, "unknown method %d", d->method);
  }
  if (mabp && (d->p < 1 || !(d->b > 0 && d->b < 1) || !(d->c > 0) || !std::isfinite(d->c) || !(d->kT > 0) ||
               !(d->w > 0) || !std::isfinite(d->w))) {
    delete w;
    return fail(ABP_ERR_INVALID_ARG, "mABP needs p >= 1, 0 < b < 1, c > 0, kT > 0 and w > 0");
  }
  if (mabp && grid->desc.shared) {
    delete w;
    return fail(ABP_ERR_UNSUPPORTED, "mABP walkers need their own grid");
  }
  hd.method = d->method;
  if (!(d->kwall >= 0) || !std::isfinite(d->kwall)) {
    delete w;
    return fail(ABP_ERR_INVALID_ARG, "kwall must be finite and >= 0");
  }
  hd.kwall = d->kwall;
  hd.kwall_f = (float)d->kwall;
  for (int k = 0; k < 3; ++k) {
    if (d->kwall > 0 && k < ncv && !std::isfinite(d->smax[k])) {
      delete w;
      return fail(ABP_ERR_INVALID_ARG, "smax[%d] must be finite when kwall > 0", k);
    }
    hd.smax[k] = d->kwall > 0 && k < ncv ? d->smax[k] : 0.0;
    hd.smax_f[k] = (float)hd.smax[k];
  }
  long long stencil = 1;
  for (int k = 0; k < ncv; ++k) {
    double sig = mabp ? d->a[k] : d->sigma[k];
    if (!(sig > 0) || !std::isfinite(sig)) {
      delete w;
      return fail(ABP_ERR_INVALID_ARG, mabp ? "a[%d] must be > 0" : "sigma[%d] must be > 0", k);
    }
    double D = spacing(grid->desc, k);
    // stencil half-width: the Gaussian's cutoff box, or the nodes within a of
    // the compact hill's centre node
    double Rd = mabp ? std::floor(sig / D) : std::ceil(d->cutoff * sig / D);
    if (Rd > kRMax) {
      delete w;
      return fail(ABP_ERR_UNSUPPORTED, "stencil half-width %g on axis %d exceeds %d nodes", Rd, k, kRMax);
    }
    hd.R[k] = (int)Rd;
    if (grid->desc.periodic[k] && 2 * hd.R[k] + 1 > grid->desc.n[k]) {
      delete w;
      return fail(ABP_ERR_INVALID_ARG, "periodic axis %d: stencil box (%d nodes) wider than the axis", k,
                  2 * hd.R[k] + 1);
    }
    hd.sigma[k] = sig;
    hd.inv2s2[k] = 1.0 / (2.0 * sig * sig);
    hd.invs2[k] = 1.0 / (sig * sig);
    hd.a[k] = mabp ? sig : 0.0;
    stencil *= 2 * hd.R[k] + 1;
  }
  hd.w = d->w;
  hd.inv_dT = mabp ? 0.0 : 1.0 / ((d->gamma - 1.0) * d->kT);
  hd.stride = d->stride;
  if (mabp) {
    hd.p = d->p;
    hd.mabp_k = d->kT * d->b / (1.0 - d->b);
    hd.mabp_g = d->c * d->b * d->kT;
    hd.mabp_h = d->c * (1.0 - d->b);
  }
  for (int k = 0; k < ncv; ++k) {
    st = build_cv(w, d->cv[k], k, d->natoms, &hd.cv[k]);
    if (st) {
      walker_free(w);
      delete w;
      return st;
    }
    if (d->cv[k].type == ABP_CV_COORD) w->has_cn = true;
    if (d->cv[k].type == ABP_CV_RMSD) w->has_rmsd = true;
    if (d->cv[k].type == ABP_CV_DIHEDRAL) hd.cv[k].hp = !fp64 && hd.sigma[k] < kDihedralHpWidth;
  }
  int rsz = fp64 ? 32 : 16;
  // the phased form serves walkers on a shared grid and walkers too large
  // for one shared-memory walker group (FP32, at most one CN)
  w->big = grid->desc.shared || run_group_bytes(hd, fp64, 32, 0, false) > 227 * 1024;
  w->win = !w->big && window_eligible(hd, fp64);
  if (w->win) {
    // the closed-loop form's a5 term tables (read, not rebuilt, by each launch)
    std::vector<int> tcnt;
    void *pc = nullptr, *pt = nullptr;
    if (fp64) {
      std::vector<AtomTerm<double>> tt;
      atom_term_tables<double>(d, ncv, tcnt, tt);
      st = upload(w, tt.data(), tt.size() * sizeof(AtomTerm<double>), &pt);
    } else {
      std::vector<AtomTerm<float>> tt;
      atom_term_tables<float>(d, ncv, tcnt, tt);
      st = upload(w, tt.data(), tt.size() * sizeof(AtomTerm<float>), &pt);
      bool fast = d->natoms <= 64;
      for (int c : tcnt) fast = fast && c <= 2;
      for (int k = 0; k < ncv; ++k)
        fast = fast && ((d->cv[k].type == ABP_CV_COM_DIST && d->cv[k].n_a <= 16 && d->cv[k].n_b <= 16) ||
                        d->cv[k].type == ABP_CV_DIHEDRAL);
      fast = fast && !mabp;
      w->md_fast = fast;
    }
    if (st == ABP_OK) st = upload(w, tcnt.data(), tcnt.size() * sizeof(int), &pc);
    if (st) {
      walker_free(w);
      delete w;
      return st;
    }
    hd.acnt = static_cast<const int *>(pc);
    hd.aterms = pt;
  }
  if ((mabp || w->has_rmsd) && w->big) {
    walker_free(w);
    delete w;
    return fail(ABP_ERR_UNSUPPORTED, "mABP and RMSD walkers run in the fused form: own grid, one SM's shared memory");
  }
  if (w->has_rmsd && !w->win) {
    walker_free(w);
    delete w;
    return fail(ABP_ERR_UNSUPPORTED, "RMSD walkers run in the windowed form (COM distance, dihedral and RMSD CVs)");
  }
  if (w->big && (fp64 || big_cn_count(hd) > 1)) {
    walker_free(w);
    delete w;
    return fail(ABP_ERR_UNSUPPORTED,
                "walkers on a shared grid or with too many atoms for one SM need FP32 grids and at most one CN");
  }
  size_t js_bytes = std::max((size_t)plain_scratch_bytes(fp64, hd.cv, ncv), w->big ? big_scratch_bytes(hd) : 0);
  void *p;
  if ((st = walker_alloc(w, (size_t)rsz * d->natoms, &p)) == ABP_OK) {
    hd.fbuf = p;
    CUDA_TRY(cudaMemset(p, 0, (size_t)rsz * d->natoms));
    if ((st = walker_alloc(w, js_bytes, &p)) == ABP_OK) {
      hd.jscratch = p;
      if ((st = walker_alloc(w, sizeof(WalkerState), &p)) == ABP_OK) {
        hd.state = static_cast<WalkerState *>(p);
        CUDA_TRY(cudaMemset(p, 0, sizeof(WalkerState)));
      }
    }
  }
  if (st == ABP_OK && w->big && big_cn_smem(hd) > 200 * 1024)
    st = fail(ABP_ERR_UNSUPPORTED, "a coordination number with more than ~2000 A atoms is not built");
  if (st == ABP_OK && w->big) {
    // the force phase's per-atom term table, into the walker's scratch
    std::vector<int32_t> terms;
    std::vector<uint8_t> cnt;
    if (big_atom_terms(hd, d, terms, cnt))
      st = fail(ABP_ERR_UNSUPPORTED, "an atom takes part in more than %d CV list entries", kAtomTerms);
    unsigned char *js = static_cast<unsigned char *>(hd.jscratch);
    if (st == ABP_OK && cudaMemcpy(js + big_terms_offset(hd), terms.data(), terms.size() * sizeof(int32_t),
                                   cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(ABP_ERR_CUDA, "term table upload failed");
    if (st == ABP_OK &&
        cudaMemcpy(js + big_nterm_offset(hd), cnt.data(), cnt.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      st = fail(ABP_ERR_CUDA, "term table upload failed");
  }
  if (st == ABP_OK) {
    hd.id = ctx->next_id++;
    if ((st = walker_alloc(w, sizeof(WalkerDev), &p)) == ABP_OK) {
      w->dd = static_cast<WalkerDev *>(p);
      CUDA_TRY(cudaMemcpy(w->dd, &hd, sizeof(WalkerDev), cudaMemcpyHostToDevice));
    }
  }
  if (st) {
    walker_free(w);
    delete w;
    return st;
  }
  long long pairs = 0;
  for (int k = 0; k < ncv; ++k)
    if (hd.cv[k].type == ABP_CV_COORD) pairs += (long long)hd.cv[k].na * hd.cv[k].nb;
  w->cost = pairs * 4 + d->natoms * 8 + stencil * 4 / d->stride;
  *out = w;
  return ABP_OK;
}

void abp_walker_destroy(abp_walker *w) {
  if (!w) return;
  std::lock_guard<std::mutex> lk(w->ctx->mu);
  set_device(w->ctx);
  cudaStreamSynchronize(w->ctx->stream);
  walker_free(w);
  delete w;
}

int32_t abp_walker_id(const abp_walker *w) { return w ? w->hd.id : -1; }

// ---------------------------------------------------------------- the force call

// Device table for a sub-list of the caller's walkers (entries keep the
// caller's index, which selects coordinate and force offsets).
static abp_status sub_table(abp_ctx *ctx, const std::vector<abp_walker *> &ws, const std::vector<int> &idx,
                            const TableEntry **out, const uint32_t *streams = nullptr) {
  // by cost, ties in list order (buffers reused: no allocation per call)
  thread_local std::vector<size_t> order;
  thread_local std::vector<TableEntry> sorted;
  order.resize(ws.size());
  for (size_t i = 0; i < ws.size(); ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return ws[a]->cost != ws[b]->cost ? ws[a]->cost > ws[b]->cost : a < b;
  });
  sorted.resize(ws.size());
  for (size_t i = 0; i < ws.size(); ++i) {
    const size_t j = order[i];
    sorted[i] = TableEntry{ws[j]->dd, idx[j], streams ? streams[idx[j]] : 0u};
  }
  ++ctx->use_clock;
  TableCache *victim = &ctx->tables[0];
  for (auto &t : ctx->tables) {
    if (t.dev && t.key.size() == sorted.size() &&
        std::memcmp(t.key.data(), sorted.data(), sorted.size() * sizeof(TableEntry)) == 0) {
      t.last_use = ctx->use_clock;
      *out = t.dev;
      return ABP_OK;
    }
    if (t.last_use < victim->last_use) victim = &t;
  }
  size_t need = std::max<size_t>(1, sorted.size()) * sizeof(TableEntry);
  if (victim->cap < need) {
    if (victim->dev) cudaFree(victim->dev);
    victim->dev = nullptr;
    victim->cap = 0;
    CUDA_TRY(cudaMalloc(&victim->dev, need));
    victim->cap = need;
  }
  CUDA_TRY(cudaMemcpyAsync(victim->dev, sorted.data(), sorted.size() * sizeof(TableEntry), cudaMemcpyHostToDevice,
                           ctx->stream));
  victim->key = sorted;
  victim->last_use = ctx->use_clock;
  *out = victim->dev;
  return ABP_OK;
}

// Items of the phased form: one per walker, then one per CN chunk.
static abp_status big_items(abp_ctx *ctx, const std::vector<abp_walker *> &ws, const std::vector<int> &idx,
                            BigArgs *a, const uint32_t *streams = nullptr) {
  std::vector<BigItem> key;
  int max_stencil = 0, any_shared = 0, max_atoms = 0;
  size_t cn_smem = 0;
  for (size_t i = 0; i < ws.size(); ++i) {
    key.push_back(BigItem{ws[i]->dd, idx[i], 0, streams ? streams[idx[i]] : 0u, 0});
    const WalkerDev &hd = ws[i]->hd;
    max_atoms = std::max(max_atoms, hd.natoms);
    int box = 1;
    for (int k = 0; k < hd.g.d; ++k) box *= 2 * hd.R[k] + 1;
    max_stencil = std::max(max_stencil, box);
    any_shared |= hd.g.shared;
    cn_smem = std::max(cn_smem, big_cn_smem(hd));
  }
  int ncn = 0;
  for (size_t i = 0; i < ws.size(); ++i) {
    int nc = big_chunks(ws[i]->hd);
    for (int c = 0; c < nc; ++c) key.push_back(BigItem{ws[i]->dd, idx[i], c, 0u, 0});
    ncn += nc;
  }
  if (key.size() != ctx->big_key.size() ||
      std::memcmp(key.data(), ctx->big_key.data(), key.size() * sizeof(BigItem)) != 0) {
    size_t need = key.size() * sizeof(BigItem);
    if (ctx->big_cap < need) {
      if (ctx->big_dev) cudaFree(ctx->big_dev);
      ctx->big_dev = nullptr;
      ctx->big_cap = 0;
      CUDA_TRY(cudaMalloc(&ctx->big_dev, need));
      ctx->big_cap = need;
    }
    CUDA_TRY(cudaMemcpyAsync(ctx->big_dev, key.data(), need, cudaMemcpyHostToDevice, ctx->stream));
    ctx->big_key = key;
  }
  a->walkers = ctx->big_dev;
  a->nw = (int)ws.size();
  a->cn_items = ctx->big_dev + ws.size();
  a->ncn_items = ncn;
  a->cn_smem = cn_smem;
  a->max_stencil = max_stencil;
  a->any_shared = any_shared;
  a->max_atoms = max_atoms;
  return ABP_OK;
}

static abp_status run_common(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords, int cdt,
                             const int64_t *coff, int64_t cstride, void *forces, const int64_t *foff,
                             int64_t fstride, int mode, int64_t step0, int nsteps) {
  int fp64;
  bool shared;
  abp_status st = check_list(ctx, walkers, n, &fp64, &shared);
  if (st) return st;
  if (shared) {
    std::set<const abp_grid *> seen;
    for (int i = 0; i < n; ++i)
      if (!seen.insert(walkers[i]->grid).second && !walkers[i]->grid->desc.shared)
        return fail(ABP_ERR_INVALID_ARG, "walkers that deposit into one grid need a grid created with shared = 1");
  }
  if (n == 0 || nsteps == 0) return ABP_OK;
  if (nsteps < 0) return fail(ABP_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (step0 < 0) return fail(ABP_ERR_INVALID_ARG, "step must be >= 0");
  if (!coords || !coff) return fail(ABP_ERR_INVALID_ARG, "coordinates or offsets are NULL");
  if (cdt != (fp64 ? ABP_F64 : ABP_F32))
    return fail(ABP_ERR_INVALID_ARG, "coordinate dtype must be %s for these walkers", fp64 ? "ABP_F64" : "ABP_F32");
  if (mode != ABP_FORCES_ACCUMULATE && mode != ABP_FORCES_OVERWRITE) return fail(ABP_ERR_INVALID_ARG, "bad mode");
  if ((reinterpret_cast<uintptr_t>(coords) & 15) || (forces && (reinterpret_cast<uintptr_t>(forces) & 15)))
    return fail(ABP_ERR_INVALID_ARG, "coordinate and force buffers must be 16-byte aligned");
  if (fp64 && ((reinterpret_cast<uintptr_t>(coords) & 31) || (forces && (reinterpret_cast<uintptr_t>(forces) & 31))))
    return fail(ABP_ERR_INVALID_ARG, "FP64 coordinate and force buffers must be 32-byte aligned");
  st = set_device(ctx);
  if (st) return st;
  // three forms: windowed (k_win, one launch per grid dimension), per-step
  // fused (k_run), phased (big)
  std::vector<abp_walker *> ww[3], fw, bw;
  std::vector<int> wi[3], fi, bi;
  for (int i = 0; i < n; ++i) {
    if (walkers[i]->big) {
      bw.push_back(walkers[i]);
      bi.push_back(i);
    } else if (walkers[i]->win) {
      ww[walkers[i]->hd.g.d - 1].push_back(walkers[i]);
      wi[walkers[i]->hd.g.d - 1].push_back(i);
    } else {
      fw.push_back(walkers[i]);
      fi.push_back(i);
    }
  }
  for (int form = 0; form < 4; ++form) {  // windowed d = 1, 2, 3, then per-step
    const bool win = form < 3;
    std::vector<abp_walker *> &lw = win ? ww[form] : fw;
    std::vector<int> &li = win ? wi[form] : fi;
    if (lw.empty()) continue;
    RunArgs a{};
    if ((st = sub_table(ctx, lw, li, &a.table))) return st;
    if ((st = pick_shape(ctx, lw.data(), (int)lw.size(), fp64, nsteps, win, &a.G, &a.groups_per_cta,
                         &a.group_bytes, &a.tile_budget)))
      return st;
    a.window = win ? form + 1 : 0;
    a.nw = (int)lw.size();
    a.lean = ctx->tune_lean && !fp64 && !win;
    a.coords = coords;
    a.coff = reinterpret_cast<const long long *>(coff);
    a.cstride = cstride;
    a.forces = forces;
    a.foff = reinterpret_cast<const long long *>(foff);
    a.fstride = fstride;
    a.mode = mode;
    a.step0 = step0;
    a.nsteps = nsteps;
    a.log = ctx->log;
    a.ctr = ctx->ctr;
    const char *kname = win ? "k_win" : (a.lean && a.tile_budget == 0 ? "k_run_lean" : "k_run");
    NvtxRange nv(kname);
    if (ctx->timer) ctx->timer->begin(kname, ctx->stream);
    cudaError_t e = launch_run(a, fp64, ctx->stream);
    if (ctx->timer) ctx->timer->end(kname, ctx->stream);
    if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "fused launch: %s", cudaGetErrorString(e));
  }
  if (!bw.empty()) {
    BigArgs b{};
    if ((st = big_items(ctx, bw, bi, &b))) return st;
    b.coords = coords;
    b.coff = reinterpret_cast<const long long *>(coff);
    b.forces = forces;
    b.foff = reinterpret_cast<const long long *>(foff);
    b.mode = mode;
    b.log = ctx->log;
    b.ctr = ctx->ctr;
    b.timer = ctx->timer;
    for (int t = 0; t < nsteps; ++t) {
      b.step = step0 + t;
      b.step_off = (long long)t * cstride;
      b.force_step_off = (long long)t * fstride;
      cudaError_t e = launch_big_step(b, ctx->stream);
      if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "phased launch: %s", cudaGetErrorString(e));
    }
  }
  return ABP_OK;
}

abp_status abp_run(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                   const int64_t *coord_offsets_dev, int64_t coord_step_stride, void *forces_dev,
                   const int64_t *force_offsets_dev, int64_t force_step_stride, int mode, int64_t step0, int nsteps) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  if (n > 0 && nsteps > 0 && (!forces_dev || !force_offsets_dev))
    return fail(ABP_ERR_INVALID_ARG, "forces or force offsets are NULL");
  return run_common(ctx, walkers, n, coords_dev, coords_dtype, coord_offsets_dev, coord_step_stride, forces_dev,
                    force_offsets_dev, force_step_stride, mode, step0, nsteps);
}

abp_status abp_md_run(abp_ctx *ctx, abp_walker *const *walkers, int n, void *coords_dev, int coords_dtype,
                      const int64_t *coord_offsets_dev, const abp_md_desc *md, const uint32_t *streams,
                      void *traj_dev, const int64_t *traj_offsets_dev, int64_t traj_step_stride, void *forces_dev,
                      const int64_t *force_offsets_dev, int64_t force_step_stride, int mode, int64_t step0,
                      int nsteps) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  int fp64;
  bool shared;
  abp_status st = check_list(ctx, walkers, n, &fp64, &shared);
  if (st) return st;
  if (shared) {
    std::set<const abp_grid *> seen;
    for (int i = 0; i < n; ++i)
      if (!seen.insert(walkers[i]->grid).second && !walkers[i]->grid->desc.shared)
        return fail(ABP_ERR_INVALID_ARG, "walkers that deposit into one grid need a grid created with shared = 1");
  }
  if (n == 0 || nsteps == 0) return ABP_OK;
  if (nsteps < 0) return fail(ABP_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (step0 < 0) return fail(ABP_ERR_INVALID_ARG, "step must be >= 0");
  if (!coords_dev || !coord_offsets_dev) return fail(ABP_ERR_INVALID_ARG, "coordinates or offsets are NULL");
  if (!md || !streams) return fail(ABP_ERR_INVALID_ARG, "dynamics descriptor or streams are NULL");
  if (traj_dev && !traj_offsets_dev) return fail(ABP_ERR_INVALID_ARG, "trajectory offsets are NULL");
  if (forces_dev && !force_offsets_dev) return fail(ABP_ERR_INVALID_ARG, "force offsets are NULL");
  if (coords_dtype != (fp64 ? ABP_F64 : ABP_F32))
    return fail(ABP_ERR_INVALID_ARG, "coordinate dtype must be %s for these walkers", fp64 ? "ABP_F64" : "ABP_F32");
  if (mode != ABP_FORCES_ACCUMULATE && mode != ABP_FORCES_OVERWRITE) return fail(ABP_ERR_INVALID_ARG, "bad mode");
  const uintptr_t amask = fp64 ? 31 : 15;
  if ((reinterpret_cast<uintptr_t>(coords_dev) & amask) || (reinterpret_cast<uintptr_t>(traj_dev) & amask) ||
      (reinterpret_cast<uintptr_t>(forces_dev) & amask))
    return fail(ABP_ERR_INVALID_ARG, "coordinate, trajectory and force buffers must be %d-byte aligned",
                (int)amask + 1);
  if (!(md->dt > 0) || !(md->mobility >= 0) || !(md->kT >= 0) || !std::isfinite(md->dt) ||
      !std::isfinite(md->mobility) || !std::isfinite(md->kT))
    return fail(ABP_ERR_INVALID_ARG, "dynamics: dt > 0, mobility >= 0 and kT >= 0 (finite) are required");
  if (md->potential < ABP_POT_NONE || md->potential > ABP_POT_MULLER_BROWN)
    return fail(ABP_ERR_INVALID_ARG, "unknown potential %d", md->potential);
  MdParams mp{};
  mp.potential = md->potential;
  mp.c1 = md->dt * md->mobility;
  mp.c2 = std::sqrt(2.0 * md->mobility * md->kT * md->dt);
  mp.seed = md->seed;
  mp.dw_a = md->dw_a;
  mp.dw_b = md->dw_b;
  mp.mb_scale = md->mb_scale;
  for (int q = 0; q < 4; ++q) {
    mp.mb_map[q] = md->mb_map[q];
    mp.mb_A[q] = md->mb_A[q];
    mp.mb_a[q] = md->mb_a[q];
    mp.mb_b[q] = md->mb_b[q];
    mp.mb_c[q] = md->mb_c[q];
    mp.mb_x0[q] = md->mb_x0[q];
    mp.mb_y0[q] = md->mb_y0[q];
  }
  if (md->potential == ABP_POT_MULLER_BROWN)
    for (int i = 0; i < n; ++i)
      if (walkers[i]->hd.g.d < 2)
        return fail(ABP_ERR_INVALID_ARG, "walker %d: the Mueller-Brown potential needs two CVs", i);
  // the one-warp form (by grid dimension) and the phased form
  thread_local std::vector<abp_walker *> ww[3], bw;  // reused: no allocation per call
  thread_local std::vector<int> wi[3], bi;
  for (int k = 0; k < 3; ++k) {
    ww[k].clear();
    wi[k].clear();
  }
  bw.clear();
  bi.clear();
  for (int i = 0; i < n; ++i) {
    if (walkers[i]->big) {
      if (md->potential != ABP_POT_NONE)
        return fail(ABP_ERR_UNSUPPORTED, "walker %d runs in the phased form, which takes no CV potential", i);
      bw.push_back(walkers[i]);
      bi.push_back(i);
    } else if (walkers[i]->win) {
      ww[walkers[i]->hd.g.d - 1].push_back(walkers[i]);
      wi[walkers[i]->hd.g.d - 1].push_back(i);
    } else {
      return fail(ABP_ERR_UNSUPPORTED,
                  "walker %d: closed-loop runs take walkers whose CVs are COM distances, dihedrals or RMSDs, and "
                  "walkers of the phased form",
                  i);
    }
  }
  if ((st = set_device(ctx))) return st;
  for (int dim = 1; dim <= 3; ++dim) {
    std::vector<abp_walker *> &lw = ww[dim - 1];
    if (lw.empty()) continue;
    MdRunArgs a{};
    if ((st = sub_table(ctx, lw, wi[dim - 1], &a.r.table, streams))) return st;
    int gb = 0;
    for (abp_walker *w : lw) gb = std::max(gb, md_group_bytes(w->hd, fp64));
    const int smem_max = 227 * 1024;
    if (gb > smem_max) return fail(ABP_ERR_UNSUPPORTED, "a walker needs %d bytes of shared memory (max %d)", gb, smem_max);
    // four warps per walker; with more walkers than multiprocessors, two
    // walker groups per CTA
    int gpc = ctx->tune_gpc ? std::min(ctx->tune_gpc, 2) : ((int)lw.size() > ctx->sms ? 2 : 1);
    while (gpc > 1 && gpc * gb > smem_max) --gpc;
    a.r.nw = (int)lw.size();
    a.r.G = 128;
    a.r.groups_per_cta = gpc;
    a.r.group_bytes = gb;
    a.r.coords = coords_dev;
    a.r.coff = reinterpret_cast<const long long *>(coord_offsets_dev);
    a.r.forces = forces_dev;
    a.r.foff = reinterpret_cast<const long long *>(force_offsets_dev);
    a.r.fstride = force_step_stride;
    a.r.mode = mode;
    a.r.step0 = step0;
    a.r.nsteps = nsteps;
    a.r.log = ctx->log;
    a.r.ctr = ctx->ctr;
    a.md = mp;
    a.traj = traj_dev;
    a.toff = reinterpret_cast<const long long *>(traj_offsets_dev);
    a.tstride = traj_step_stride;
    bool fast = !fp64;
    for (abp_walker *w : lw) fast = fast && w->md_fast;
    NvtxRange nv("k_md");
    if (ctx->timer) ctx->timer->begin("k_md", ctx->stream);
    cudaError_t e = launch_md(a, fp64, dim, fast, ctx->stream);
    if (ctx->timer) ctx->timer->end("k_md", ctx->stream);
    if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "closed-loop launch: %s", cudaGetErrorString(e));
  }
  if (!bw.empty()) {
    BigArgs b{};
    if ((st = big_items(ctx, bw, bi, &b, streams))) return st;
    b.coords = coords_dev;
    b.coff = reinterpret_cast<const long long *>(coord_offsets_dev);
    b.forces = forces_dev;
    b.foff = reinterpret_cast<const long long *>(force_offsets_dev);
    b.mode = mode;
    b.log = ctx->log;
    b.ctr = ctx->ctr;
    b.md = &mp;
    b.timer = ctx->timer;
    b.xio = coords_dev;
    b.traj = traj_dev;
    b.toff = reinterpret_cast<const long long *>(traj_offsets_dev);
    for (int t = 0; t < nsteps; ++t) {
      b.step = step0 + t;
      b.step_off = 0;  // the coordinates stay where they are and move in place
      b.force_step_off = (long long)t * force_step_stride;
      b.traj_step_off = (long long)t * traj_step_stride;
      cudaError_t e = launch_big_step(b, ctx->stream);
      if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "phased launch: %s", cudaGetErrorString(e));
    }
  }
  return ABP_OK;
}

abp_status abp_step(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                    const int64_t *coord_offsets_dev, int64_t step) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  return run_common(ctx, walkers, n, coords_dev, coords_dtype, coord_offsets_dev, 0, nullptr, nullptr, 0,
                    ABP_FORCES_OVERWRITE, step, 1);
}

abp_status abp_forces(abp_ctx *ctx, abp_walker *const *walkers, int n, void *forces_dev, int forces_dtype,
                      const int64_t *force_offsets_dev, int mode) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  int fp64;
  bool shared;
  abp_status st = check_list(ctx, walkers, n, &fp64, &shared);
  if (st) return st;
  if (n == 0) return ABP_OK;
  if (!forces_dev || !force_offsets_dev) return fail(ABP_ERR_INVALID_ARG, "forces or offsets are NULL");
  if (forces_dtype != (fp64 ? ABP_F64 : ABP_F32)) return fail(ABP_ERR_INVALID_ARG, "force dtype mismatch");
  if (mode != ABP_FORCES_ACCUMULATE && mode != ABP_FORCES_OVERWRITE) return fail(ABP_ERR_INVALID_ARG, "bad mode");
  if ((st = set_device(ctx))) return st;
  const TableEntry *table;
  if ((st = get_table(ctx, walkers, n, false, &table))) return st;
  cudaError_t e = launch_deliver(table, n, forces_dev, reinterpret_cast<const long long *>(force_offsets_dev), mode,
                                 fp64, ctx->stream);
  if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "force delivery: %s", cudaGetErrorString(e));
  return ABP_OK;
}

abp_status abp_step_plain(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                          const int64_t *coord_offsets_dev, void *forces_dev, const int64_t *force_offsets_dev,
                          int mode, int64_t step) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  int fp64;
  bool shared;
  abp_status st = check_list(ctx, walkers, n, &fp64, &shared);
  if (st) return st;
  if (shared) return fail(ABP_ERR_UNSUPPORTED, "the plain form takes walkers with their own grids");
  for (int i = 0; i < n; ++i)
    if (walkers[i]->big || walkers[i]->has_rmsd)
      return fail(ABP_ERR_UNSUPPORTED, "walker %d runs only in the batched form (shared grid, too many atoms or RMSD)",
                  i);
  if (n == 0) return ABP_OK;
  if (step < 0) return fail(ABP_ERR_INVALID_ARG, "step must be >= 0");
  if (!coords_dev || !coord_offsets_dev || !forces_dev || !force_offsets_dev)
    return fail(ABP_ERR_INVALID_ARG, "NULL buffer");
  if (coords_dtype != (fp64 ? ABP_F64 : ABP_F32)) return fail(ABP_ERR_INVALID_ARG, "coordinate dtype mismatch");
  if (mode != ABP_FORCES_ACCUMULATE && mode != ABP_FORCES_OVERWRITE) return fail(ABP_ERR_INVALID_ARG, "bad mode");
  if ((st = set_device(ctx))) return st;
  std::vector<const WalkerDev *> wd(n);
  std::vector<int> dyn(n), dep(n);
  const int threads = 128;
  for (int i = 0; i < n; ++i) {
    wd[i] = walkers[i]->dd;
    dyn[i] = dyn_bytes(walkers[i], threads / 32);
    dep[i] = (step % walkers[i]->hd.stride) == 0;
  }
  PlainArgs a{};
  a.nw = n;
  a.wd_dev = wd.data();
  a.dyn_bytes = dyn.data();
  a.deposit = dep.data();
  a.threads = threads;
  a.coords = coords_dev;
  a.coff = reinterpret_cast<const long long *>(coord_offsets_dev);
  a.forces = forces_dev;
  a.foff = reinterpret_cast<const long long *>(force_offsets_dev);
  a.mode = mode;
  a.step = step;
  a.log = ctx->log;
  a.ctr = ctx->ctr;
  NvtxRange nv("plain form");
  cudaError_t e = launch_plain(a, fp64, ctx->stream);
  if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "plain launch: %s", cudaGetErrorString(e));
  return ABP_OK;
}

// ---------------------------------------------------------------- hill exchange

namespace {

// Walkers of an exchange call: all in the phased form on shared grids.
abp_status exchange_list(abp_ctx *ctx, abp_walker *const *walkers, int n) {
  int fp64;
  bool shared;
  abp_status st = check_list(ctx, walkers, n, &fp64, &shared);
  if (st) return st;
  for (int i = 0; i < n; ++i)
    if (!walkers[i]->grid->desc.shared)
      return fail(ABP_ERR_INVALID_ARG, "walker %d: hill exchange needs a grid created with shared = 1", i);
  return ABP_OK;
}

// Grid-index position of a hill centre on axis k, as the deposit places it
// (non-periodic centres clamped like the deposit's guard).
double hill_axis(const abp_walker *w, int k, double s) {
  const GridDev &g = w->hd.g;
  const int n = g.n[k], R = w->hd.R[k];
  double x = (s - g.lo[k]) * g.invD[k];
  if (g.periodic[k]) return x - std::floor(x / n) * n;
  return std::min(std::max(x, (double)(-R - 2)), (double)(n + R + 1));
}

// Whether the stencil boxes of two hills may share a node. A box spans
// centre +- R nodes and a centre lies within 1/2 node (plus float-float
// rounding) of the position u, so positions more than 2R + 2 apart on some
// axis give disjoint boxes.
bool boxes_may_overlap(const abp_walker *w, const double *ua, const double *ub) {
  const GridDev &g = w->hd.g;
  for (int k = 0; k < g.d; ++k) {
    const double reach = 2.0 * w->hd.R[k] + 2.0;
    double dist = std::fabs(ua[k] - ub[k]);
    if (g.periodic[k]) {
      const int n = g.n[k];
      if (2 * w->hd.R[k] + 3 >= n) continue;  // a box that spans the axis meets every other
      dist = std::min(dist, n - dist);
    }
    if (dist > reach) return false;
  }
  return true;
}

}  // namespace

abp_status abp_shared_hills(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                            const int64_t *coord_offsets_dev, int64_t step, abp_hill *hills_out, size_t cap,
                            size_t *n_out) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  if (n_out) *n_out = 0;
  abp_status st = exchange_list(ctx, walkers, n);
  if (st) return st;
  if (n == 0) return ABP_OK;
  if (step < 0) return fail(ABP_ERR_INVALID_ARG, "step must be >= 0");
  if (!coords_dev || !coord_offsets_dev || !n_out) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  if (coords_dtype != ABP_F32) return fail(ABP_ERR_INVALID_ARG, "coordinate dtype must be ABP_F32");
  if (reinterpret_cast<uintptr_t>(coords_dev) & 15)
    return fail(ABP_ERR_INVALID_ARG, "coordinate buffer must be 16-byte aligned");
  if ((st = set_device(ctx))) return st;
  std::vector<abp_walker *> ws(walkers, walkers + n);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  BigArgs b{};
  if ((st = big_items(ctx, ws, idx, &b))) return st;
  b.coords = coords_dev;
  b.coff = reinterpret_cast<const long long *>(coord_offsets_dev);
  b.mode = ABP_FORCES_OVERWRITE;
  b.log = ctx->log;
  b.ctr = ctx->ctr;
  b.step = step;
  b.phases = 1 | 2;
  cudaError_t e = launch_big_step(b, ctx->stream);
  if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "hill phase: %s", cudaGetErrorString(e));
  std::vector<const WalkerDev *> hd(n);
  for (int i = 0; i < n; ++i) hd[i] = &walkers[i]->hd;
  std::vector<double> s3h(4 * (size_t)n);
  std::vector<int> dep(n);
  e = read_hill_heads(hd.data(), n, s3h.data(), dep.data(), ctx->stream);
  if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "hill readout: %s", cudaGetErrorString(e));
  size_t m = 0;
  for (int i = 0; i < n; ++i) {
    if (!dep[i]) continue;
    if (m < cap && hills_out) {
      abp_hill &h = hills_out[m];
      for (int k = 0; k < 3; ++k) h.s[k] = k < walkers[i]->hd.g.d ? s3h[4 * i + k] : 0.0;
      h.height = s3h[4 * i + 3];
      h.step = step;
      h.walker_id = walkers[i]->hd.id;
      h.pad = 0;
    }
    ++m;
  }
  *n_out = m;
  if (m > cap || (m > 0 && !hills_out))
    return fail(ABP_ERR_INVALID_ARG, "%zu hills but room for %zu", m, hills_out ? cap : (size_t)0);
  return ABP_OK;
}

abp_status abp_grid_apply_hills(abp_ctx *ctx, const abp_walker *shape, const abp_hill *hills, size_t n) {
  if (!ctx || !shape) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  if (shape->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "walker belongs to another context");
  if (!shape->grid->desc.shared) return fail(ABP_ERR_INVALID_ARG, "hill records apply to grids created with shared = 1");
  if (n == 0) return ABP_OK;
  if (!hills) return fail(ABP_ERR_INVALID_ARG, "hills is NULL");
  if (n > (1u << 24)) return fail(ABP_ERR_INVALID_ARG, "too many hill records");
  const int d = shape->hd.g.d;
  std::vector<double> u(3 * n, 0.0);
  for (size_t j = 0; j < n; ++j) {
    if (!std::isfinite(hills[j].height) || hills[j].height < 0)
      return fail(ABP_ERR_INVALID_ARG, "hill %zu: height must be finite and >= 0", j);
    for (int k = 0; k < d; ++k) {
      if (!std::isfinite(hills[j].s[k])) return fail(ABP_ERR_INVALID_ARG, "hill %zu: centre is not finite", j);
      u[3 * j + k] = hill_axis(shape, k, hills[j].s[k]);
    }
  }
  // wave of record j: one past the last wave holding an earlier record whose
  // box may meet j's, so every node receives its hills in list order
  std::vector<int> wave(n, 0);
  int nwaves = 0;
  for (size_t j = 0; j < n; ++j) {
    int w = 0;
    for (size_t i = 0; i < j; ++i)
      if (wave[i] >= w && boxes_may_overlap(shape, &u[3 * i], &u[3 * j])) w = wave[i] + 1;
    wave[j] = w;
    nwaves = std::max(nwaves, w + 1);
  }
  std::vector<HillDev> recs;
  std::vector<int> start(nwaves + 1, 0);
  recs.reserve(n);
  for (int w = 0; w < nwaves; ++w) {
    start[w] = (int)recs.size();
    for (size_t j = 0; j < n; ++j)
      if (wave[j] == w) {
        HillDev h;
        for (int k = 0; k < 3; ++k) h.s[k] = k < d ? hills[j].s[k] : 0.0;
        h.h = hills[j].height;
        recs.push_back(h);
      }
  }
  start[nwaves] = (int)recs.size();
  abp_status st = set_device(ctx);
  if (st) return st;
  const size_t need = recs.size() * sizeof(HillDev);
  if (ctx->hill_cap < need) {
    if (ctx->hill_dev) cudaFree(ctx->hill_dev);
    ctx->hill_dev = nullptr;
    ctx->hill_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->hill_dev, need));
    ctx->hill_cap = need;
  }
  CUDA_TRY(cudaMemcpyAsync(ctx->hill_dev, recs.data(), need, cudaMemcpyHostToDevice, ctx->stream));
  int box = 1;
  for (int k = 0; k < d; ++k) box *= 2 * shape->hd.R[k] + 1;
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < nwaves && e == cudaSuccess; ++w)
    e = launch_apply_hills(shape->dd, ctx->hill_dev + start[w], start[w + 1] - start[w], box, false, ctx->stream);
  if (e == cudaSuccess) e = launch_apply_hills(shape->dd, ctx->hill_dev, (int)recs.size(), box, true, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the host records may go once this returns
  if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "hill apply: %s", cudaGetErrorString(e));
  return ABP_OK;
}

abp_status abp_shared_forces(abp_ctx *ctx, abp_walker *const *walkers, int n, void *forces_dev, int forces_dtype,
                             const int64_t *force_offsets_dev, int mode, int64_t step) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  abp_status st = exchange_list(ctx, walkers, n);
  if (st) return st;
  if (n == 0) return ABP_OK;
  if (!forces_dev || !force_offsets_dev) return fail(ABP_ERR_INVALID_ARG, "forces or offsets are NULL");
  if (forces_dtype != ABP_F32) return fail(ABP_ERR_INVALID_ARG, "force dtype must be ABP_F32");
  if (reinterpret_cast<uintptr_t>(forces_dev) & 15) return fail(ABP_ERR_INVALID_ARG, "force buffer must be 16-byte aligned");
  if (mode != ABP_FORCES_ACCUMULATE && mode != ABP_FORCES_OVERWRITE) return fail(ABP_ERR_INVALID_ARG, "bad mode");
  if ((st = set_device(ctx))) return st;
  std::vector<abp_walker *> ws(walkers, walkers + n);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  BigArgs b{};
  if ((st = big_items(ctx, ws, idx, &b))) return st;
  b.forces = forces_dev;
  b.foff = reinterpret_cast<const long long *>(force_offsets_dev);
  b.mode = mode;
  b.step = step;
  b.phases = 16;
  cudaError_t e = launch_big_step(b, ctx->stream);
  if (e != cudaSuccess) return fail(ABP_ERR_CUDA, "force phase: %s", cudaGetErrorString(e));
  return ABP_OK;
}

// ---------------------------------------------------------------- readouts

size_t abp_grid_record_bytes(const abp_grid *g) { return g ? g->bytes + g->shadow_bytes : 0; }

abp_status abp_grid_save(abp_ctx *ctx, const abp_grid *g, void *dst, int dst_is_device) {
  if (!ctx || !g || !dst || g->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "bad argument");
  abp_status st = set_device(ctx);
  if (st) return st;
  const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpyAsync(dst, g->g.rec, g->bytes, kind, ctx->stream));
  if (g->shadow_bytes)
    CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned char *>(dst) + g->bytes, g->g.shadow, g->shadow_bytes, kind,
                             ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ABP_OK;
}

abp_status abp_grid_restore(abp_ctx *ctx, abp_grid *g, const void *src, int src_is_device) {
  if (!ctx || !g || !src || g->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "bad argument");
  abp_status st = set_device(ctx);
  if (st) return st;
  const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(g->g.rec, src, g->bytes, kind, ctx->stream));
  if (g->shadow_bytes)
    CUDA_TRY(cudaMemcpyAsync(g->g.shadow, static_cast<const unsigned char *>(src) + g->bytes, g->shadow_bytes, kind,
                             ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  return ABP_OK;
}

abp_status abp_bias_readout(abp_ctx *ctx, const abp_grid *g, void *dst, int dst_is_device, int dtype) {
  if (!ctx || !g || !dst || g->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "bad argument");
  if (dtype != ABP_F32 && dtype != ABP_F64) return fail(ABP_ERR_INVALID_ARG, "bad dtype");
  abp_status st = set_device(ctx);
  if (st) return st;
  const GridDev &gd = g->g;
  const int d = gd.d, nf = 1 + d;
  std::vector<unsigned char> raw(g->bytes);
  CUDA_TRY(cudaMemcpyAsync(raw.data(), gd.rec, g->bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const size_t nvals = (size_t)gd.nodes * nf;
  std::vector<double> v(nvals);
  for (long long i = 0; i < gd.nodes; ++i) {
    for (int q = 0; q < nf; ++q) {
      double x;
      if (gd.prec == ABP_PREC_FP32_COMP) {
        const float *r = reinterpret_cast<const float *>(raw.data() + (size_t)i * gd.rec_bytes);
        int comp_off = d == 1 ? 2 : 4;
        x = (double)r[q] + (double)r[comp_off + q];
      } else {
        x = reinterpret_cast<const double *>(raw.data() + (size_t)i * gd.rec_bytes)[q];
      }
      v[(size_t)i * nf + q] = x;
    }
  }
  const void *src = v.data();
  std::vector<float> vf;
  size_t bytes = nvals * sizeof(double);
  if (dtype == ABP_F32) {
    vf.resize(nvals);
    for (size_t i = 0; i < nvals; ++i) vf[i] = (float)v[i];
    src = vf.data();
    bytes = nvals * sizeof(float);
  }
  if (dst_is_device) {
    CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return ABP_OK;
}

abp_status abp_bias_upload(abp_ctx *ctx, abp_grid *g, const void *src, int src_is_device, int dtype) {
  if (!ctx || !g || !src || g->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "bad argument");
  if (dtype != ABP_F32 && dtype != ABP_F64) return fail(ABP_ERR_INVALID_ARG, "bad dtype");
  abp_status st = set_device(ctx);
  if (st) return st;
  const GridDev &gd = g->g;
  const int d = gd.d, nf = 1 + d;
  const size_t nvals = (size_t)gd.nodes * nf;
  const size_t esz = dtype == ABP_F64 ? 8 : 4;
  std::vector<unsigned char> in(nvals * esz);
  if (src_is_device) {
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    CUDA_TRY(cudaMemcpy(in.data(), src, in.size(), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(in.data(), src, in.size());
  }
  std::vector<unsigned char> raw(g->bytes, 0);
  for (long long i = 0; i < gd.nodes; ++i) {
    for (int q = 0; q < nf; ++q) {
      size_t j = (size_t)i * nf + q;
      double x = dtype == ABP_F64 ? reinterpret_cast<const double *>(in.data())[j]
                                  : (double)reinterpret_cast<const float *>(in.data())[j];
      if (gd.prec == ABP_PREC_FP32_COMP) {
        float *r = reinterpret_cast<float *>(raw.data() + (size_t)i * gd.rec_bytes);
        int comp_off = d == 1 ? 2 : 4;
        float hi = (float)x;
        r[q] = hi;
        r[comp_off + q] = (float)(x - (double)hi);
      } else {
        reinterpret_cast<double *>(raw.data() + (size_t)i * gd.rec_bytes)[q] = x;
      }
    }
  }
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(cudaMemcpy(gd.rec, raw.data(), g->bytes, cudaMemcpyHostToDevice));
  if (gd.shadow) {
    // a shared grid's accumulator takes the exact values
    std::vector<double> sh((size_t)gd.nodes * 4, 0.0);
    for (long long i = 0; i < gd.nodes; ++i)
      for (int q = 0; q < nf; ++q) {
        size_t j = (size_t)i * nf + q;
        sh[(size_t)i * 4 + q] = dtype == ABP_F64 ? reinterpret_cast<const double *>(in.data())[j]
                                                 : (double)reinterpret_cast<const float *>(in.data())[j];
      }
    CUDA_TRY(cudaMemcpy(gd.shadow, sh.data(), sh.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  return ABP_OK;
}

abp_status abp_walker_readout(abp_ctx *ctx, const abp_walker *w, double *s, double *V, double *dV, int *flags) {
  if (!ctx || !w || w->ctx != ctx) return fail(ABP_ERR_INVALID_ARG, "bad argument");
  abp_status st = set_device(ctx);
  if (st) return st;
  WalkerState hs;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(cudaMemcpy(&hs, w->hd.state, sizeof hs, cudaMemcpyDeviceToHost));
  for (int k = 0; k < 3; ++k) {
    if (s) s[k] = hs.s[k];
    if (dV) dV[k] = hs.dV[k];
  }
  if (V) *V = hs.V;
  if (flags) *flags = hs.flags;
  if (hs.flags & ABP_WFLAG_NONFINITE) return fail(ABP_ERR_NONFINITE, "the walker's last step saw non-finite coordinates");
  return ABP_OK;
}

abp_status abp_deposit_log_enable(abp_ctx *ctx, size_t capacity) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  abp_status st = set_device(ctx);
  if (st) return st;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (ctx->log.rec) cudaFree(ctx->log.rec);
  if (ctx->log.count) cudaFree(ctx->log.count);
  ctx->log = DepositLog{nullptr, nullptr, 0};
  if (capacity == 0) return ABP_OK;
  CUDA_TRY(cudaMalloc(&ctx->log.rec, capacity * sizeof(abp_deposit_rec)));
  CUDA_TRY(cudaMalloc(&ctx->log.count, sizeof(unsigned long long)));
  CUDA_TRY(cudaMemset(ctx->log.count, 0, sizeof(unsigned long long)));
  ctx->log.cap = capacity;
  return ABP_OK;
}

abp_status abp_deposit_log_readout(abp_ctx *ctx, abp_deposit_rec *dst, size_t cap, size_t *n_out, size_t *n_total) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  abp_status st = set_device(ctx);
  if (st) return st;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  unsigned long long cnt = 0;
  if (ctx->log.count) CUDA_TRY(cudaMemcpy(&cnt, ctx->log.count, sizeof cnt, cudaMemcpyDeviceToHost));
  size_t stored = (size_t)std::min<unsigned long long>(cnt, ctx->log.cap);
  size_t n = std::min(stored, cap);
  if (n && !dst) return fail(ABP_ERR_INVALID_ARG, "dst is NULL");
  if (n) CUDA_TRY(cudaMemcpy(dst, ctx->log.rec, n * sizeof(abp_deposit_rec), cudaMemcpyDeviceToHost));
  if (n_out) *n_out = n;
  if (n_total) *n_total = (size_t)cnt;
  return ABP_OK;
}

abp_status abp_deposit_log_clear(abp_ctx *ctx) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  abp_status st = set_device(ctx);
  if (st) return st;
  if (ctx->log.count) CUDA_TRY(cudaMemsetAsync(ctx->log.count, 0, sizeof(unsigned long long), ctx->stream));
  return ABP_OK;
}

abp_status abp_sync(abp_ctx *ctx) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  abp_status st = set_device(ctx);
  if (st) return st;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  int nf = 0;
  CUDA_TRY(cudaMemcpy(&nf, &ctx->ctr->nonfinite, sizeof nf, cudaMemcpyDeviceToHost));
  if (nf) {
    CUDA_TRY(cudaMemset(&ctx->ctr->nonfinite, 0, sizeof nf));
    return fail(ABP_ERR_NONFINITE, "%d walker steps saw non-finite coordinates", nf);
  }
  return ABP_OK;
}

}  // extern "C"

// ===================================================================== serving
//
// abp_server: continuous batching of single-step requests from many
// simulations. The server owns nstreams "slots" (stream, two events, pinned
// and device buffers for coordinates, forces, offsets, per-walker steps and
// the walker table) and two threads:
//   the launcher fills a free slot with the front request of every
//   simulation that has one (FIFO, one request per simulation and slot, up
//   to max_batch), packs it and launches the fused kernel for one step on
//   the slot's stream. A simulation whose previous request is still on the
//   GPU in another slot goes into the new slot too: the new slot's kernel
//   waits on the device for that slot's kernel (an event), so the steps of
//   one simulation run in order while the host works ahead;
//   the deliverer takes launched slots in launch order (so one simulation's
//   results come back in step order), waits for each, copies its forces to
//   the callers' buffers and frees the slot.
// Packing the next slot, the GPU and delivering the previous slot overlap.

#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <memory>
#include <thread>
#include <atomic>
#include <unordered_map>

namespace {

// A fixed team of helper threads for the host copies of a large launch:
// run(fn) calls fn(part, nparts) for every part, part 0 on the calling
// thread, and returns when all parts are done.
class CopyTeam {
 public:
  explicit CopyTeam(int helpers) : nparts_(helpers + 1) {
    for (int i = 0; i < helpers; ++i) threads_.emplace_back([this, i] { loop(i + 1); });
  }
  ~CopyTeam() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : threads_) t.join();
  }
  void run(const std::function<void(int, int)> &fn) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      left_ = nparts_ - 1;
      ++gen_;
    }
    cv_.notify_all();
    fn(0, nparts_);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return left_ == 0; });
    fn_ = nullptr;
  }

 private:
  void loop(int part) {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(int, int)> *fn;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        fn = fn_;
      }
      (*fn)(part, nparts_);
      std::lock_guard<std::mutex> lk(mu_);
      if (--left_ == 0) done_.notify_one();
    }
  }
  const int nparts_;
  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int, int)> *fn_ = nullptr;
  int left_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// Requests [lo, hi) of part p of np, split so that each part copies about
// the same number of atoms (off: the requests' atom offsets, total atoms).
void part_range(const long long *off, int n, long long total, int p, int np, int *lo, int *hi) {
  auto first_at = [&](long long atom) { return (int)(std::lower_bound(off, off + n, atom) - off); };
  *lo = first_at(total * p / np);
  *hi = p + 1 == np ? n : first_at(total * (p + 1) / np);
}

constexpr long long kTeamAtoms = 16384;  // below this a launch is copied by one thread
constexpr double kLauncherSpin = 50e-6;   // seconds the launcher spins for work before it sleeps

double steady_now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvSim;

struct SrvRequest {
  int64_t sim = 0, step = 0;
  uint64_t tag = 0;
  float *forces_host = nullptr;
  double t_submit = 0;
  std::shared_ptr<std::vector<float>> slab;  // the coordinates' storage (shared by one submit call)
  const float *coords = nullptr;             // natoms records inside slab
  int natoms = 0;
  SrvSim *simp = nullptr;  // stable while the request is queued or in flight
};

struct SrvSim {
  abp_grid *grid = nullptr;
  abp_walker *walker = nullptr;
  int natoms = 0;
  std::deque<SrvRequest> pending;
  int inflight = 0;     // requests in slots not yet delivered
  int last_slot = -1;   // the slot holding its newest request in flight
  bool in_ready = false;
  int gb_g[2] = {0, 0}, gb[2] = {0, 0};  // group bytes cached for two group sizes
};

struct SrvSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t kdone = nullptr;  // after the slot's kernel
  cudaEvent_t done = nullptr;   // after the forces are back in pinned memory
  // h_in / d_in: one upload per launch, the coordinates followed by the
  // walker table, the offsets and the steps of the batch (contiguous for
  // the batch's sizes); h_off / h_step / h_table point into h_in for the
  // batch in the slot
  float *h_in = nullptr, *h_out = nullptr;
  long long *h_off = nullptr, *h_step = nullptr;
  TableEntry *h_table = nullptr;
  float *d_in = nullptr, *d_out = nullptr;
  std::vector<SrvRequest> reqs;
  std::vector<abp_walker *> ws;
  std::vector<int> deps;  // slots whose kernels this slot's kernel waits for
  bool cn = false;        // a walker with a coordination number is in the slot
  int G = 0, gb = 0;      // group size and the largest group footprint at G
  bool busy = false;
  int status = ABP_OK;
};

}  // namespace

struct abp_server {
  abp_ctx *ctx = nullptr;
  int max_batch = 4096, max_atoms = 1024, nstreams = 2;
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_launched;
  // bumped after every change that cv_work announces: the launcher spins on
  // it for a while before it sleeps
  std::atomic<unsigned long long> work_seq{0};
  std::unordered_map<int64_t, SrvSim> sims;
  int64_t next_sim = 0;
  std::deque<int64_t> ready;  // simulations with pending requests (each once)
  std::deque<abp_result> results;
  std::vector<SrvSlot> slots;
  std::deque<int> launched;  // slots in flight, in launch order
  std::thread launcher, deliverer;
  bool stop = false, stop_delivery = false;
  int64_t submitted = 0, finished = 0, launches = 0, queued = 0;
  // thread seconds by phase (each written under mu by its thread)
  double t_fill = 0, t_launch = 0, t_complete = 0, t_wait = 0;
  // coordinate slabs of delivered requests, kept for reuse (their pages
  // stay mapped: a fresh multi-megabyte copy would fault every page in)
  std::mutex pool_mu;
  std::vector<std::vector<float> *> slab_pool;
  // helper teams for the launcher's packing and the deliverer's unpacking
  std::unique_ptr<CopyTeam> pack_team, unpack_team;
};

namespace {

void srv_free_slots(abp_server *s) {
  for (auto &sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaFreeHost(sl.h_in);
    cudaFreeHost(sl.h_out);
    cudaFree(sl.d_in);
    cudaFree(sl.d_out);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.kdone) cudaEventDestroy(sl.kdone);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  s->slots.clear();
}

// A copy of n floats from src in a slab from the pool (the smallest that
// holds them, else a new one); the slab returns to the pool when the last
// request using it is gone. Lock order: mu, then pool_mu.
std::shared_ptr<std::vector<float>> srv_slab(abp_server *s, const float *src, size_t n) {
  std::vector<float> *v = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->pool_mu);
    size_t best = s->slab_pool.size();
    for (size_t i = 0; i < s->slab_pool.size(); ++i)
      if (s->slab_pool[i]->capacity() >= n &&
          (best == s->slab_pool.size() || s->slab_pool[i]->capacity() < s->slab_pool[best]->capacity()))
        best = i;
    if (best < s->slab_pool.size()) {
      v = s->slab_pool[best];
      s->slab_pool[best] = s->slab_pool.back();
      s->slab_pool.pop_back();
    }
  }
  if (!v) v = new std::vector<float>();
  v->assign(src, src + n);
  return std::shared_ptr<std::vector<float>>(v, [s](std::vector<float> *p) {
    // small slabs come from the heap's free lists without faults: only the
    // large ones (one submit_many chunk) are kept
    if (p->capacity() * sizeof(float) >= (256u << 10)) {
      std::lock_guard<std::mutex> lk(s->pool_mu);
      if (s->slab_pool.size() < 64) {
        s->slab_pool.push_back(p);
        return;
      }
    }
    delete p;
  });
}

// A simulation's group footprint at g threads per group (cached: the walker
// does not change while it is admitted).
int srv_group_bytes(SrvSim &sm, int g) {
  for (int i = 0; i < 2; ++i)
    if (sm.gb_g[i] == g) return sm.gb[i];
  const int b = run_group_bytes(sm.walker->hd, 0, g, 0, false);
  const int i = sm.gb_g[0] ? 1 : 0;
  sm.gb_g[i] = g;
  sm.gb[i] = b;
  return b;
}

// Pack and launch the requests now in the slot (launcher thread, without the
// server lock; the slot's walkers and shape were taken under it).
int srv_launch(abp_server *s, SrvSlot &sl) {
  const int n = (int)sl.reqs.size();
  // the batch's walker table, offsets and steps are written behind its
  // coordinates in the upload buffer, so that one copy takes them all
  long long total = 0;
  for (int i = 0; i < n; ++i) total += sl.reqs[i].natoms;
  const size_t tab_at = (size_t)total * 16, off_at = tab_at + (size_t)n * sizeof(TableEntry),
               step_at = off_at + (size_t)n * 8, upload = step_at + (size_t)n * 8;
  unsigned char *hb = reinterpret_cast<unsigned char *>(sl.h_in);
  unsigned char *db = reinterpret_cast<unsigned char *>(sl.d_in);
  sl.h_table = reinterpret_cast<TableEntry *>(hb + tab_at);
  sl.h_off = reinterpret_cast<long long *>(hb + off_at);
  sl.h_step = reinterpret_cast<long long *>(hb + step_at);
  long long off = 0;
  for (int i = 0; i < n; ++i) {
    const SrvRequest &r = sl.reqs[i];
    sl.h_off[i] = off;
    sl.h_step[i] = r.step;
    sl.h_table[i] = TableEntry{sl.ws[i]->dd, i, 0};
    off += r.natoms;
  }
  auto pack = [&](int p, int np) {
    int lo, hi;
    part_range(sl.h_off, n, off, p, np, &lo, &hi);
    for (int i = lo; i < hi; ++i)
      std::memcpy(sl.h_in + sl.h_off[i] * 4, sl.reqs[i].coords, (size_t)sl.reqs[i].natoms * 16);
  };
  if (off >= kTeamAtoms && s->pack_team)
    s->pack_team->run(pack);
  else
    pack(0, 1);
  RunArgs a{};
  int st = step_shape(s->ctx, sl.cn, sl.G, sl.gb, 0, &a.G, &a.groups_per_cta, &a.group_bytes, &a.tile_budget);
  if (st) return st;
  cudaStream_t stream = sl.stream;
  if (cudaMemcpyAsync(db, hb, upload, cudaMemcpyHostToDevice, stream) != cudaSuccess) return ABP_ERR_CUDA;
  const TableEntry *d_table = reinterpret_cast<const TableEntry *>(db + tab_at);
  const long long *d_off = reinterpret_cast<const long long *>(db + off_at);
  const long long *d_step = reinterpret_cast<const long long *>(db + step_at);
  // the previous step of a simulation in this slot runs in another slot:
  // its kernel (grid deposit, walker state) must finish first
  for (int d : sl.deps)
    if (cudaStreamWaitEvent(stream, s->slots[d].kdone, 0) != cudaSuccess) return ABP_ERR_CUDA;
  a.table = d_table;
  a.nw = n;
  a.coords = sl.d_in;
  a.coff = d_off;
  a.cstride = 0;
  a.forces = sl.d_out;
  a.foff = d_off;
  a.fstride = 0;
  a.mode = ABP_FORCES_OVERWRITE;
  a.step0 = 0;
  a.wstep = d_step;
  a.nsteps = 1;
  a.log = s->ctx->log;
  a.ctr = s->ctx->ctr;
  {
    NvtxRange nv("server launch");
    if (launch_run(a, 0, stream) != cudaSuccess) return ABP_ERR_CUDA;
  }
  if (cudaEventRecord(sl.kdone, stream) != cudaSuccess) return ABP_ERR_CUDA;
  if (cudaMemcpyAsync(sl.h_out, sl.d_out, (size_t)off * 16, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return ABP_ERR_CUDA;
  if (cudaEventRecord(sl.done, stream) != cudaSuccess) return ABP_ERR_CUDA;
  return ABP_OK;
}

// Deliver a finished slot's requests (deliverer thread, without the lock).
void srv_complete(abp_server *s, SrvSlot &sl) {
  const int n = (int)sl.reqs.size();
  if (sl.status == ABP_OK && n > 0) {
    const long long total = sl.h_off[n - 1] + sl.reqs[n - 1].natoms;
    auto unpack = [&](int p, int np) {
      int lo, hi;
      part_range(sl.h_off, n, total, p, np, &lo, &hi);
      for (int i = lo; i < hi; ++i)
        std::memcpy(sl.reqs[i].forces_host, sl.h_out + sl.h_off[i] * 4, (size_t)sl.reqs[i].natoms * 16);
    };
    if (total >= kTeamAtoms && s->unpack_team)
      s->unpack_team->run(unpack);
    else
      unpack(0, 1);
  }
  const double t = steady_now();  // the forces are in the callers' buffers
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = 0; i < n; ++i) {
      const SrvRequest &r = sl.reqs[i];
      s->results.push_back(abp_result{r.sim, r.step, r.tag, r.t_submit, t, sl.status, n});
      --r.simp->inflight;
    }
    s->finished += n;
    sl.reqs.clear();
    sl.ws.clear();
    sl.deps.clear();
    sl.busy = false;
  }
  s->cv_done.notify_all();
  s->work_seq.fetch_add(1, std::memory_order_release);
  s->cv_work.notify_one();  // a slot is free
}

// Fill slot fi from the ready simulations (server lock held): one request
// per simulation; simulations with more requests stay ready for the next
// slot.
void srv_fill(abp_server *s, int fi) {
  SrvSlot &sl = s->slots[fi];
  const abp_ctx *ctx = s->ctx;
  int atoms = 0;
  std::vector<SrvSim *> again;
  sl.cn = false;
  while (!s->ready.empty() && (int)sl.reqs.size() < s->max_batch) {
    auto it = s->sims.find(s->ready.front());
    if (it == s->sims.end()) {
      s->ready.pop_front();
      continue;
    }
    SrvSim &sm = it->second;
    if (sm.pending.empty()) {
      s->ready.pop_front();
      sm.in_ready = false;
      continue;
    }
    if (atoms + sm.natoms > s->max_batch * s->max_atoms) break;
    s->ready.pop_front();
    sm.in_ready = false;
    if (sm.inflight > 0) sl.deps.push_back(sm.last_slot);
    ++sm.inflight;
    sm.last_slot = fi;
    atoms += sm.natoms;
    sl.cn = sl.cn || sm.walker->has_cn;
    sl.reqs.push_back(std::move(sm.pending.front()));
    sl.ws.push_back(sm.walker);
    sm.pending.pop_front();
    --s->queued;
    if (!sm.pending.empty()) again.push_back(&sm);
  }
  for (SrvSim *sm : again) {
    s->ready.push_back(sm->pending.front().sim);
    sm->in_ready = true;
  }
  std::sort(sl.deps.begin(), sl.deps.end());
  sl.deps.erase(std::unique(sl.deps.begin(), sl.deps.end()), sl.deps.end());
  // the launch shape: the per-step form's group size for this mix, and the
  // largest footprint at that size
  sl.G = ctx->tune_G ? ctx->tune_G : (sl.cn ? 128 : 32);
  sl.gb = 0;
  for (const SrvRequest &r : sl.reqs) sl.gb = std::max(sl.gb, srv_group_bytes(*r.simp, sl.G));
  sl.busy = !sl.reqs.empty();
}

void srv_launcher(abp_server *s) {
  cudaSetDevice(s->ctx->device);
  double t_fill = 0, t_launch = 0;
  for (;;) {
    int fi = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->t_fill = t_fill;
      s->t_launch = t_launch;
      auto free_slot = [&] {
        for (int i = 0; i < (int)s->slots.size(); ++i)
          if (!s->slots[i].busy) return i;
        return -1;
      };
      auto work = [&] { return s->stop || (!s->ready.empty() && free_slot() >= 0); };
      if (!work()) {
        // spin for up to kLauncherSpin seconds before sleeping: a request (or
        // a freed slot) that comes within it is taken without a thread wake-up
        const unsigned long long seq0 = s->work_seq.load(std::memory_order_acquire);
        lk.unlock();
        const double t_spin = steady_now();
        for (int it = 0; s->work_seq.load(std::memory_order_acquire) == seq0; ++it)
          if ((it & 255) == 255 && steady_now() - t_spin > kLauncherSpin) break;
        lk.lock();
      }
      s->cv_work.wait(lk, work);
      if (s->stop) break;
      const double t0 = steady_now();
      fi = free_slot();
      srv_fill(s, fi);
      t_fill += steady_now() - t0;
      if (!s->slots[fi].busy) continue;
    }
    const double t1 = steady_now();
    SrvSlot &sl = s->slots[fi];
    sl.status = srv_launch(s, sl);
    if (sl.status != ABP_OK) {
      // the slot still goes to the deliverer in launch order; record its
      // events so that it and any slot queued after it on the device end
      cudaGetLastError();
      cudaEventRecord(sl.kdone, sl.stream);
      cudaEventRecord(sl.done, sl.stream);
      cudaGetLastError();
    }
    t_launch += steady_now() - t1;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->launched.push_back(fi);
      ++s->launches;
    }
    s->cv_launched.notify_one();
  }
}

void srv_deliverer(abp_server *s) {
  cudaSetDevice(s->ctx->device);
  double t_complete = 0, t_wait = 0;
  for (;;) {
    int fi;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->t_complete = t_complete;
      s->t_wait = t_wait;
      s->cv_launched.wait(lk, [&] { return !s->launched.empty() || s->stop_delivery; });
      if (s->launched.empty()) break;
      fi = s->launched.front();
    }
    SrvSlot &sl = s->slots[fi];
    const double t0 = steady_now();
    cudaError_t q = cudaEventSynchronize(sl.done);
    const double t1 = steady_now();
    t_wait += t1 - t0;
    if (q != cudaSuccess) {
      cudaGetLastError();
      sl.status = ABP_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->launched.pop_front();
    }
    srv_complete(s, sl);
    t_complete += steady_now() - t1;
  }
}

}  // namespace

extern "C" {

double abp_server_now(void) { return steady_now(); }

abp_status abp_server_create(abp_ctx *ctx, const abp_server_desc *desc, abp_server **out) {
  if (!ctx || !out) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  abp_server *s = new (std::nothrow) abp_server();
  if (!s) return fail(ABP_ERR_OOM, "host allocation failed");
  s->ctx = ctx;
  if (desc) {
    if (desc->max_batch < 0 || desc->max_atoms < 0 || desc->nstreams < 0 || desc->nstreams > 8) {
      delete s;
      return fail(ABP_ERR_INVALID_ARG, "bad server descriptor");
    }
    if (desc->max_batch) s->max_batch = desc->max_batch;
    if (desc->max_atoms) s->max_atoms = desc->max_atoms;
    if (desc->nstreams) s->nstreams = desc->nstreams;
  }
  abp_status st = set_device(ctx);
  if (st) {
    delete s;
    return st;
  }
  const size_t rec = (size_t)s->max_batch * s->max_atoms * 16;
  const size_t meta = (size_t)s->max_batch * (sizeof(TableEntry) + 16);  // table, offsets, steps
  s->slots.resize(s->nstreams);
  cudaError_t e = cudaSuccess;
  for (auto &sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.kdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_in, rec + meta, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_out, rec, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_in, rec + meta);
    if (e == cudaSuccess) e = cudaMalloc(&sl.d_out, rec);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    srv_free_slots(s);
    delete s;
    return fail(ABP_ERR_OOM, "server buffers: %s", cudaGetErrorString(e));
  }
  // two helpers each for packing and unpacking where the host has the cores
  const unsigned hw = std::thread::hardware_concurrency();
  if (hw >= 8) {
    s->pack_team.reset(new CopyTeam(2));
    s->unpack_team.reset(new CopyTeam(2));
  }
  s->launcher = std::thread(srv_launcher, s);
  s->deliverer = std::thread(srv_deliverer, s);
  *out = s;
  return ABP_OK;
}

void abp_server_destroy(abp_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->work_seq.fetch_add(1, std::memory_order_release);
  s->cv_work.notify_all();
  if (s->launcher.joinable()) s->launcher.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_delivery = true;  // the deliverer finishes the launched slots first
  }
  s->cv_launched.notify_all();
  if (s->deliverer.joinable()) s->deliverer.join();
  set_device(s->ctx);
  srv_free_slots(s);
  for (auto &kv : s->sims) {
    abp_walker_destroy(kv.second.walker);
    abp_grid_destroy(kv.second.grid);
  }
  s->sims.clear();  // queued requests return their slabs to the pool
  for (std::vector<float> *p : s->slab_pool) delete p;
  s->slab_pool.clear();
  delete s;
}

abp_status abp_server_admit(abp_server *s, const abp_grid_desc *g, const abp_walker_desc *w, int64_t *sim) {
  if (!s || !g || !w || !sim) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  if (g->shared) return fail(ABP_ERR_UNSUPPORTED, "the server takes walkers on their own grids");
  if (g->precision != ABP_PREC_FP32_COMP) return fail(ABP_ERR_UNSUPPORTED, "the server serves FP32_COMP grids");
  if (w->natoms > s->max_atoms) return fail(ABP_ERR_INVALID_ARG, "walker has more atoms than max_atoms");
  abp_grid *grid = nullptr;
  abp_status st = abp_create_grid(s->ctx, g, &grid);
  if (st) return st;
  abp_walker *walker = nullptr;
  st = abp_walker_create(s->ctx, grid, w, &walker);
  if (st) {
    std::string msg = g_err;
    abp_grid_destroy(grid);
    return fail(st, "%s", msg.c_str());
  }
  if (walker->big || walker->has_rmsd) {
    abp_walker_destroy(walker);
    abp_grid_destroy(grid);
    return fail(ABP_ERR_UNSUPPORTED, "the server serves walkers that fit one walker group (no RMSD CVs)");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t id = s->next_sim++;
  SrvSim &sm = s->sims[id];
  sm.grid = grid;
  sm.walker = walker;
  sm.natoms = w->natoms;
  *sim = id;
  return ABP_OK;
}

abp_status abp_server_bias_readout(abp_server *s, int64_t sim, void *dst, int dst_is_device, int dtype) {
  if (!s || !dst) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  abp_grid *grid = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->sims.find(sim);
    if (it == s->sims.end()) return fail(ABP_ERR_INVALID_ARG, "unknown simulation %lld", (long long)sim);
    if (!s->cv_done.wait_for(lk, std::chrono::seconds(60), [&] {
          auto jt = s->sims.find(sim);
          return jt == s->sims.end() || (jt->second.inflight == 0 && jt->second.pending.empty());
        }))
      return fail(ABP_ERR_TIMEOUT, "simulation %lld still has requests after 60 s", (long long)sim);
    it = s->sims.find(sim);
    if (it == s->sims.end()) return fail(ABP_ERR_INVALID_ARG, "simulation %lld was released", (long long)sim);
    grid = it->second.grid;
  }
  return abp_bias_readout(s->ctx, grid, dst, dst_is_device, dtype);
}

abp_status abp_server_release(abp_server *s, int64_t sim) {
  if (!s) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  SrvSim sm;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->sims.find(sim);
    if (it == s->sims.end()) return fail(ABP_ERR_INVALID_ARG, "unknown simulation %lld", (long long)sim);
    if (!s->cv_done.wait_for(lk, std::chrono::seconds(60), [&] {
          auto jt = s->sims.find(sim);
          return jt == s->sims.end() || (jt->second.inflight == 0 && jt->second.pending.empty());
        }))
      return fail(ABP_ERR_TIMEOUT, "simulation %lld still has requests after 60 s", (long long)sim);
    it = s->sims.find(sim);
    sm = std::move(it->second);
    s->sims.erase(it);
  }
  abp_walker_destroy(sm.walker);
  abp_grid_destroy(sm.grid);
  return ABP_OK;
}

abp_status abp_server_submit(abp_server *s, int64_t sim, int64_t step, const float *coords_host, float *forces_host,
                             uint64_t tag) {
  if (!s || !coords_host || !forces_host) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  if (step < 0) return fail(ABP_ERR_INVALID_ARG, "step must be >= 0");
  SrvRequest r;
  r.sim = sim;
  r.step = step;
  r.tag = tag;
  r.forces_host = forces_host;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->sims.find(sim);
    if (it == s->sims.end()) return fail(ABP_ERR_INVALID_ARG, "unknown simulation %lld", (long long)sim);
    SrvSim &sm = it->second;
    r.natoms = sm.natoms;
    r.simp = &sm;
    r.slab = std::make_shared<std::vector<float>>(coords_host, coords_host + (size_t)sm.natoms * 4);
    r.coords = r.slab->data();
    r.t_submit = steady_now();
    sm.pending.push_back(std::move(r));
    if (!sm.in_ready) {
      s->ready.push_back(sim);
      sm.in_ready = true;
    }
    ++s->submitted;
    ++s->queued;
  }
  s->work_seq.fetch_add(1, std::memory_order_release);
  s->cv_work.notify_one();
  return ABP_OK;
}

abp_status abp_server_submit_many(abp_server *s, int n, const int64_t *sims, const int64_t *steps,
                                  const float *coords_host, float *forces_host, const uint64_t *tags) {
  if (!s || n < 0 || (n > 0 && (!sims || !steps || !coords_host || !forces_host)))
    return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  const double t = steady_now();
  std::vector<int> nat(n);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int k = 0; k < n; ++k) {
      auto it = s->sims.find(sims[k]);
      if (it == s->sims.end()) return fail(ABP_ERR_INVALID_ARG, "unknown simulation %lld", (long long)sims[k]);
      if (steps[k] < 0) return fail(ABP_ERR_INVALID_ARG, "step must be >= 0");
      nat[k] = it->second.natoms;
    }
  }
  // queued in chunks, each copied outside the lock, so that the launcher
  // starts on the first chunk while the later ones are copied
  constexpr int kChunk = 2048;
  size_t off = 0;
  for (int k0 = 0; k0 < n; k0 += kChunk) {
    const int k1 = std::min(n, k0 + kChunk);
    size_t total = 0;
    for (int k = k0; k < k1; ++k) total += (size_t)nat[k];
    auto slab = srv_slab(s, coords_host + off * 4, total * 4);
    std::vector<SrvRequest> reqs(k1 - k0);
    size_t o = 0;
    for (int k = k0; k < k1; ++k) {
      SrvRequest &r = reqs[k - k0];
      r.sim = sims[k];
      r.step = steps[k];
      r.tag = tags ? tags[k] : 0;
      r.forces_host = forces_host + (off + o) * 4;
      r.natoms = nat[k];
      r.slab = slab;
      r.coords = slab->data() + o * 4;
      r.t_submit = t;
      o += (size_t)nat[k];
    }
    off += total;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (int k = k0; k < k1; ++k)
        if (s->sims.find(sims[k]) == s->sims.end())
          return fail(ABP_ERR_INVALID_ARG, "simulation %lld was released during the call", (long long)sims[k]);
      for (int k = k0; k < k1; ++k) {
        SrvSim &sm = s->sims[sims[k]];
        SrvRequest &r = reqs[k - k0];
        r.simp = &sm;
        sm.pending.push_back(std::move(r));
        if (!sm.in_ready) {
          s->ready.push_back(sims[k]);
          sm.in_ready = true;
        }
      }
      s->submitted += k1 - k0;
      s->queued += k1 - k0;
    }
    s->work_seq.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_one();
  }
  return ABP_OK;
}

abp_status abp_checked_violations(abp_ctx *ctx, uint64_t *count, int *checked) {
  if (!ctx) return fail(ABP_ERR_INVALID_ARG, "ctx is NULL");
  abp_status st = set_device(ctx);
  if (st) return st;
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  unsigned long long n = 0;
  CUDA_TRY(cudaMemcpy(&n, &ctx->ctr->oob, sizeof n, cudaMemcpyDeviceToHost));
  if (count) *count = (uint64_t)n;
#ifdef ABP_CHECKED
  if (checked) *checked = 1;
#else
  if (checked) *checked = 0;
#endif
  return ABP_OK;
}

abp_status abp_server_cancel(abp_server *s, int64_t sim, int64_t *n_cancelled) {
  if (!s) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  int64_t n = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->sims.find(sim);
    if (it == s->sims.end()) return fail(ABP_ERR_INVALID_ARG, "unknown simulation %lld", (long long)sim);
    SrvSim &sm = it->second;
    const double t = steady_now();
    for (const SrvRequest &r : sm.pending)
      s->results.push_back(abp_result{r.sim, r.step, r.tag, r.t_submit, t, ABP_ERR_CANCELLED, 0});
    n = (int64_t)sm.pending.size();
    sm.pending.clear();  // the ready queue skips a simulation with nothing pending
    s->queued -= n;
    s->finished += n;
  }
  if (n) s->cv_done.notify_all();
  if (n_cancelled) *n_cancelled = n;
  return ABP_OK;
}

abp_status abp_server_poll(abp_server *s, abp_result *out, int cap, int *n_out, int wait_ms) {
  if (!s || !n_out || (cap > 0 && !out)) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->results.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->results.empty(); });
  int n = 0;
  while (n < cap && !s->results.empty()) {
    out[n++] = s->results.front();
    s->results.pop_front();
  }
  *n_out = n;
  return ABP_OK;
}

abp_status abp_server_times(abp_server *s, double *fill_s, double *launch_s, double *complete_s, double *wait_s) {
  if (!s) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (fill_s) *fill_s = s->t_fill;
  if (launch_s) *launch_s = s->t_launch;
  if (complete_s) *complete_s = s->t_complete;
  if (wait_s) *wait_s = s->t_wait;
  return ABP_OK;
}

abp_status abp_server_stats(abp_server *s, int64_t *submitted, int64_t *finished, int64_t *launches, int64_t *queued) {
  if (!s) return fail(ABP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (submitted) *submitted = s->submitted;
  if (finished) *finished = s->finished;
  if (launches) *launches = s->launches;
  if (queued) *queued = s->queued;
  return ABP_OK;
}

}  // extern "C"
