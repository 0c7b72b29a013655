// abp_launch.h -- launch descriptors between the host ABI layer and the
// kernel translation units.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "abp_internal.cuh"

namespace abp {

// An NVTX range named after the kernel around each of the library's launches
// (header-only NVTX: a no-op unless a profiler attaches), so that a timeline
// or an NVTX-filtered ncu capture finds the launches by name.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Optional per-kernel timing of a context (abp_ctx_tune ABP_TUNE_TIMING): the
// launchers bracket each kernel launch with begin/end, which record CUDA
// events on the launch's stream (read back by abp_kernel_times).
struct LaunchTimer {
  virtual void begin(const char *kernel, cudaStream_t st) = 0;
  virtual void end(const char *kernel, cudaStream_t st) = 0;
  virtual ~LaunchTimer() = default;
};

// One walker of a batched launch: its device descriptor and its index in
// the caller's walker list (which selects its coordinate/force offsets).
struct TableEntry {
  const WalkerDev *wd;
  int idx;
  unsigned stream;  // the walker's noise stream in a closed-loop launch (0 otherwise)
};

struct RunArgs {
  const TableEntry *table;
  int nw;
  int G;               // threads per walker group
  int groups_per_cta;
  int group_bytes;     // shared memory per group (fixed + dynamic part)
  const void *coords;
  const long long *coff;
  long long cstride;   // records between consecutive steps
  void *forces;        // NULL: write each walker's own force buffer (abp_step)
  const long long *foff;
  long long fstride;
  int mode;
  long long step0;
  const long long *wstep;  // optional: per-walker first step (indexed like coff), overrides step0
  int nsteps;
  int tile_budget;     // >0: dynamic shared bytes per group, the rest of which holds a grid tile
  int lean;            // use the 128-register instantiation (FP32, no tile)
  int window;          // d > 0: every walker has d CVs and runs in the windowed form (k_win)
  DepositLog log;
  DevCounters *ctr;
};

struct PlainArgs {
  int nw;
  const WalkerDev *const *wd_dev;  // host array of device descriptors
  const int *dyn_bytes;            // host array: dynamic smem per walker
  const int *deposit;              // host array: deposit this step?
  int threads;
  const void *coords;
  const long long *coff;
  void *forces;
  const long long *foff;
  int mode;
  long long step;
  DepositLog log;
  DevCounters *ctr;
};

// One work item of the phased form: a walker (and, for the pair kernel, one
// chunk of its coordination-number B list).
struct BigItem {
  const WalkerDev *wd;
  int widx;
  int chunk;
  unsigned stream;  // walker items of a closed-loop call: the walker's noise stream
  int pad;
};

struct BigArgs {
  const BigItem *cn_items;
  int ncn_items;
  size_t cn_smem;
  const BigItem *walkers;
  int nw;
  const void *coords;
  const long long *coff;
  long long step_off;        // records: step t of a multi-step call
  void *forces;              // NULL: the walkers' own force buffers (abp_step)
  const long long *foff;
  long long force_step_off;
  int mode;
  long long step;
  int max_stencil;           // largest stencil box (nodes) among the walkers
  int max_atoms;             // most atoms of a walker (the force phase's CTAs per walker)
  int any_shared;
  int phases;                // bits: 1 pairs, 2 CVs + heights, 4 deposit, 8 refresh, 16 forces (0 = all)
  LaunchTimer *timer;        // per-kernel timing (NULL: off)
  const MdParams *md;        // closed loop: the force phase also moves the atoms (NULL: open loop)
  void *xio;                 // closed loop: the coordinates, moved in place
  void *traj;                // closed loop: records of the coordinates each step was evaluated at (or NULL)
  const long long *toff;
  long long traj_step_off;
  DepositLog log;
  DevCounters *ctr;
};

// A closed-loop launch (abp_md_run): the batched arguments (coords is
// written in place), the dynamics, and the optional trajectory records.
struct MdRunArgs {
  RunArgs r;
  MdParams md;
  void *traj;               // NULL: not recorded
  const long long *toff;
  long long tstride;
};

// Closed-loop form of walkers whose CVs a thread evaluates (abp_md.cu).
int md_group_bytes(const WalkerDev &hd, int fp64);
cudaError_t launch_md(const MdRunArgs &a, int fp64, int dim, bool fast, cudaStream_t st);

size_t big_scratch_bytes(const WalkerDev &hd);
// The force phase's per-atom term table of a phased-form walker (host side;
// uploaded into its scratch): per atom, codes kind | k << 3 | position << 5
// in the order a5 adds them. Returns -1 if an atom has more than kAtomTerms.
int big_atom_terms(const WalkerDev &hd, const abp_walker_desc *d, std::vector<int32_t> &terms,
                   std::vector<uint8_t> &cnt);
size_t big_terms_offset(const WalkerDev &hd);
size_t big_nterm_offset(const WalkerDev &hd);
int big_cn_count(const WalkerDev &hd);
int big_chunks(const WalkerDev &hd);
size_t big_cn_smem(const WalkerDev &hd);
cudaError_t launch_big_step(const BigArgs &a, cudaStream_t st);
// Hill records handed to a grid: one per record, in waves of disjoint boxes.
struct HillDev {
  double s[3];
  double h;
};
cudaError_t launch_apply_hills(const WalkerDev *shape, const HillDev *recs, int n, int max_stencil, bool refresh,
                               cudaStream_t st);
// Read back each walker's hill record of the last CVs + heights phase.
cudaError_t read_hill_heads(const WalkerDev *const *wd_host, int n, double *s3h, int *dep, cudaStream_t st);

int group_fixed_bytes(int fp64);
int plain_scratch_bytes(int fp64, const CvDev *cv, int ncv);
int run_group_bytes(const WalkerDev &hd, int fp64, int G, int tile_budget, bool window);
bool window_eligible(const WalkerDev &hd, int fp64);
cudaError_t launch_run(const RunArgs &a, int fp64, cudaStream_t st);
cudaError_t launch_plain(const PlainArgs &a, int fp64, cudaStream_t st);
// Records `msg` as the calling thread's abp_last_error() and returns code.
abp_status record_error(abp_status code, const char *msg);
// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) unless fn was
// already given at least that many bytes on the current device: a driver
// call on every launch otherwise.
cudaError_t smem_attr(const void *fn, size_t bytes);
cudaError_t launch_deliver(const TableEntry *table, int nw, void *forces, const long long *foff, int mode, int fp64,
                           cudaStream_t st);

}  // namespace abp
