/*
 * abp.h -- C ABI of the GB300 adaptive-biasing-potential (ABP) force call.
 *
 * The library implements, on one GPU, the per-MD-step bias routine of
 * Dickson et al., "A fast, open source implementation of adaptive biasing
 * potentials ..." (arXiv:1609.09833): it receives only the coordinates of
 * the atoms that enter the collective variables (CVs) and returns the bias
 * force on those atoms, which the owner adds to its MD force (SI,
 * "Minimization of Interprocess Communications"). Per walker and MD step:
 *
 *   a1  CVs s_k(x): centre-of-mass distance, dihedral, coordination number;
 *   a2  on a deposit step (step % stride == 0) the well-tempered height
 *       h = w exp(-V_b(s_t) / ((gamma-1) kT)) from the grid before the
 *       deposit (one exponential per hill, "Timing of the implementation",
 *       WTmetaD paragraph);
 *   a3  deposit of h exp(-|xi - s_t|^2 / 2 sigma^2) and of its derivative
 *       along each CV on the grid points of a cutoff box around s_t (value
 *       and derivative fields as in Eq. (histos), updated as in Eq. (update)
 *       over a neighbourhood of the trajectory as in Eq. (Cupdate));
 *   a4  V_b(s_t) and dV_b/ds_k(s_t) by multilinear interpolation of the value
 *       field and of each derivative field (the histogram look-up after
 *       Eq. (ghill));
 *   a5  F = - sum_k dV_b/ds_k ds_k/dx on every CV atom.
 *
 * Conventions (all calls):
 *   - Every function returns abp_status: ABP_OK (0) or a negative error
 *     code; abp_last_error() returns a thread-local message for the last
 *     failure of the calling thread. No C++ exception, abort or exit crosses
 *     this boundary.
 *   - Pointers named *_dev are device pointers on the context's GPU; the
 *     caller owns them and keeps them valid until the call's work has run on
 *     the context stream. Descriptor structs and their host arrays are read
 *     during the call only. Handles (abp_ctx, abp_grid, abp_walker) are owned
 *     by the library and freed by the matching destroy call.
 *   - Coordinates and forces are 4-component records per atom
 *     (x, y, z, pad), float (ABP_F32) or double (ABP_F64), in nm and
 *     kJ/mol/nm. Walker w's atom i at MD step t of a call is record
 *     coord_offsets_dev[w] + t * coord_step_stride + i.
 *   - Compute calls are asynchronous on the context stream; readouts and
 *     abp_sync wait for it.
 *   - Units: nm, kJ/mol, rad.
 */
#ifndef ABP_H
#define ABP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int abp_status;

#define ABP_OK 0
#define ABP_ERR_INVALID_ARG (-1)  /* a bad pointer, size, descriptor or mix of walkers */
#define ABP_ERR_CUDA (-2)         /* a CUDA runtime call failed (message says which) */
#define ABP_ERR_OOM (-3)          /* device allocation failed */
#define ABP_ERR_ADMISSION (-4)    /* the allocation would exceed the context's HBM budget */
#define ABP_ERR_NONFINITE (-5)    /* non-finite coordinates were seen; those walkers were left unchanged */
#define ABP_ERR_TIMEOUT (-6)      /* a bounded device or host wait ran out */
#define ABP_ERR_UNSUPPORTED (-7)  /* a combination the library does not implement */
#define ABP_ERR_CANCELLED (-8)    /* a served request was cancelled before it was launched */

/* CV types (step a1). */
#define ABP_CV_COM_DIST 0 /* |R_B - R_A|, R_G the mass-weighted centre of group G */
#define ABP_CV_DIHEDRAL 1 /* IUPAC dihedral of idx_a[0..3], in [-pi, pi] */
#define ABP_CV_COORD 2    /* sum over A x B of (1 - (r/r0)^n) / (1 - (r/r0)^m); n = 6, m = 12 */
#define ABP_CV_RMSD 3     /* (sum_i |x_i - x0_i|^2 / n_a + 0.01)^(1/2) over idx_a, no fit (SI "Definition of the
                             RMSD"); n_a <= 4; runs in the batched (windowed) form only */

/* Biasing methods (abp_walker_desc.method). */
#define ABP_METHOD_WT 0   /* well-tempered Gaussian hills, multilinear look-up (the default) */
#define ABP_METHOD_MABP 1 /* mABP with compact S_a^p hills at the nearest node (SI "Streamlined bias
                             potential updates"): the grid holds the histograms h and dh/dxi_k of
                             Eqs. (histos)/(Cupdate); the force uses Eq. (btraj-grad) at the nearest
                             node; not available to walkers on a shared grid */

/* Grid precision. */
#define ABP_PREC_FP32_COMP 0 /* FP32 fields with a two-sum compensation term per field */
#define ABP_PREC_FP64 1      /* FP64 fields (and FP64 CV arithmetic, FP64 coordinates) */

/* Element types for coordinate, force and readout buffers. */
#define ABP_F32 0
#define ABP_F64 1

/* Force delivery modes. */
#define ABP_FORCES_ACCUMULATE 0 /* forces[i] += bias force (the owner's MD force array) */
#define ABP_FORCES_OVERWRITE 1  /* forces[i]  = bias force */

/* Walker flags reported by abp_walker_readout. */
#define ABP_WFLAG_DEPOSIT 1   /* this step deposited a hill */
#define ABP_WFLAG_OOR 2       /* a CV was outside a non-periodic grid range (clamped) */
#define ABP_WFLAG_SINGULAR 4  /* a CV Jacobian was undefined; its gradient was set to 0 */
#define ABP_WFLAG_NONFINITE 8 /* non-finite coordinates: step skipped, state unchanged */

typedef struct abp_ctx abp_ctx;
typedef struct abp_grid abp_grid;
typedef struct abp_walker abp_walker;

/* Grid over ncv = 1..3 CVs. Nodes: non-periodic axis xi_i = lo + i D,
 * D = (hi - lo) / (n - 1), i = 0..n-1; periodic axis D = (hi - lo) / n with
 * wrap-around. Fields per node: V and dV/dxi_k for k < ncv. Node index
 * i0 + n0 (i1 + n1 i2) (axis 0 fastest). */
typedef struct {
  int ncv;
  int n[3];
  int periodic[3];
  double lo[3];
  double hi[3];
  int precision; /* ABP_PREC_* */
  int shared;    /* nonzero: several walkers deposit here in the same step; an
                    FP64 accumulator shadow receives every hill (atomics) and the
                    FP32 fields are refreshed from it (FP32_COMP grids only) */
} abp_grid_desc;

/* One CV over the walker's own block of natoms atoms. Index arrays are
 * host arrays of atom indices in [0, natoms). */
typedef struct {
  int type;              /* ABP_CV_* */
  int n_a, n_b;          /* COM: group sizes; DIHEDRAL: n_a = 4, n_b = 0; COORD: |A|, |B| */
  const int32_t *idx_a;  /* COM group A, the 4 dihedral atoms, or CN group A */
  const int32_t *idx_b;  /* COM group B or CN group B (NULL when n_b = 0) */
  const double *mass_a;  /* COM masses (NULL = unit masses); ignored otherwise */
  const double *mass_b;
  double r0;             /* COORD switching radius (nm) */
  int nn, mm;            /* COORD exponents; nn = 6, mm = 12 are supported */
  int pbc;               /* minimum image on difference vectors (orthorhombic box) */
  double box[3];
  const double *ref;     /* RMSD: reference positions of the atoms idx_a, 3 n_a values (host) */
} abp_cv_desc;

/* A walker: its atoms, one CV per grid axis and its hills. A zeroed tail
 * (method = ABP_METHOD_WT) describes a well-tempered walker. */
typedef struct {
  int natoms;
  abp_cv_desc cv[3];     /* cv[k] drives grid axis k; the grid's ncv are used */
  double w;              /* WT: initial hill height (kJ/mol); mABP: the height of every hill (1 in the paper) */
  double sigma[3];       /* WT: Gaussian width per CV */
  double cutoff;         /* WT: half-width R_k = ceil(cutoff sigma_k / D_k) of the stencil box, in sigma */
  double gamma;          /* WT: bias factor (> 1) */
  double kT;             /* thermal energy (kJ/mol); beta^-1 of Eq. (apfm) */
  int64_t stride;        /* deposit when step % stride == 0 */
  int method;            /* ABP_METHOD_* */
  double a[3];           /* mABP: compact hill half-width per CV (CV units); stencil half-width floor(a_k / D_k) */
  int p;                 /* mABP: compact hill shape exponent, >= 1 (Eq. (compacthill)) */
  double b, c;           /* mABP: the parameters of Eq. (apfm), 0 < b < 1, c > 0 */
  double smax[3];        /* CV range limit (the restraint "which limits the maximum value of the CVs",
                            Applications section; the paper gives no form): a harmonic wall */
  double kwall;          /* kwall/2 (s_k - smax_k)^2 above smax_k, added to dV_b/ds_k for the forces
                            (walker readouts report the sum); 0 = no wall */
} abp_walker_desc;

/* One deposited hill (the deposit log). */
typedef struct {
  int64_t step;
  int32_t walker_id;     /* abp_walker_id() of the walker */
  int32_t ic[3];         /* centre node index per axis, floor(u + 1/2) wrapped on periodic axes */
  double s[3];           /* s_t as computed on the device */
  double height;         /* h (FP64) */
} abp_deposit_rec;

/* ---- context ------------------------------------------------------------ */

/* Creates a context on `device`, issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). hbm_budget_bytes caps the
 * bytes the context may allocate for grids and walkers (0 = no cap): an
 * allocation beyond it fails with ABP_ERR_ADMISSION. */
abp_status abp_ctx_create(abp_ctx **out, int device, void *cuda_stream, size_t hbm_budget_bytes);
abp_status abp_ctx_set_stream(abp_ctx *ctx, void *cuda_stream);
/* Bytes currently allocated against the budget. */
abp_status abp_ctx_bytes(const abp_ctx *ctx, size_t *used, size_t *budget);

/* Launch-shape knobs of the batched form, for the autotuner, and the timing
 * switch (the paper has no counterpart: its bias routine runs on one CPU
 * rank). 0 (or -1 for ABP_TUNE_TILE) restores the library's default choice. Knobs change only
 * the schedule: results are bit-identical for every tile setting and every
 * number of groups per CTA; a different group width changes the order of
 * the CV sums, so results then agree to rounding.
 *   ABP_TUNE_GROUP_THREADS   threads per walker group: 32, 64, 128 or 256
 *   ABP_TUNE_GROUPS_PER_CTA  walker groups per CTA: 1..8
 *   ABP_TUNE_TILE            1 = give groups a shared-memory tile of their
 *                            grid when it fits (launches of >= 8 steps),
 *                            0 or -1 = never (the default)
 *   ABP_TUNE_LEAN            1 = FP32 launches without a tile use the
 *                            kernel compiled for 128 registers per thread
 *                            (two 256-thread CTAs per SM), 0 = the default
 * Invalid values return ABP_ERR_INVALID_ARG and leave the knob unchanged. */
#define ABP_TUNE_GROUP_THREADS 1
#define ABP_TUNE_GROUPS_PER_CTA 2
#define ABP_TUNE_TILE 3
#define ABP_TUNE_LEAN 4
#define ABP_TUNE_TIMING 5 /* 1 = bracket every kernel launch of the context with CUDA events (read by
                             abp_kernel_times); 0 = off (the default). Changes no result. */
abp_status abp_ctx_tune(abp_ctx *ctx, int knob, int value);

/* Per-kernel device time of the context's launches since the last call
 * (with ABP_TUNE_TIMING on): up to cap entries {kernel name, launches,
 * milliseconds summed over the launches}; *n_out receives the count. Syncs
 * the context stream; the totals restart after the call. With timing off,
 * *n_out = 0. Launches captured into a CUDA graph are not timed. */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
} abp_kernel_time;
abp_status abp_kernel_times(abp_ctx *ctx, abp_kernel_time *out, int cap, int *n_out);
void abp_ctx_destroy(abp_ctx *ctx);

/* ---- grids and walkers ---------------------------------------------------- */

/* Allocates a zeroed bias grid (V = 0 everywhere, the paper's initial
 * condition after Eq. (update)). Grid points must number >= 2 per axis. */
abp_status abp_create_grid(abp_ctx *ctx, const abp_grid_desc *desc, abp_grid **out);
void abp_grid_destroy(abp_grid *grid);
/* Zeroes every field again. */
abp_status abp_grid_clear(abp_ctx *ctx, abp_grid *grid);

/* Creates a walker depositing into `grid` (several walkers may share one
 * grid; see abp_step for the ordering). Rejects a periodic stencil box wider
 * than its axis (2R+1 > n), indices outside [0, natoms), and unsupported CV
 * parameters, with ABP_ERR_INVALID_ARG. */
abp_status abp_walker_create(abp_ctx *ctx, abp_grid *grid, const abp_walker_desc *desc, abp_walker **out);
void abp_walker_destroy(abp_walker *walker);
int32_t abp_walker_id(const abp_walker *walker);

/* ---- the force call --------------------------------------------------------- */

/* One MD step `step` for n walkers (steps a1..a5). The bias force of each
 * walker is kept in a library-owned buffer until abp_forces delivers it.
 * coords_dev: 4-component records (dtype ABP_F32 for FP32_COMP grids,
 * ABP_F64 for FP64 grids); coord_offsets_dev: n device int64 record offsets.
 * All walkers of one call must have grids of the same precision. Walkers that
 * share a grid take their heights from the grid before any deposit of the
 * step and read V_b after all of them, deposits being applied in list order
 * (Jacobi order); walkers with their own grids are independent. */
abp_status abp_step(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                    const int64_t *coord_offsets_dev, int64_t step);

/* Delivers the forces of the last abp_step of each walker into forces_dev
 * (records at force_offsets_dev[w] + i, dtype as coords), by mode. */
abp_status abp_forces(abp_ctx *ctx, abp_walker *const *walkers, int n, void *forces_dev, int forces_dtype,
                      const int64_t *force_offsets_dev, int mode);

/* The fused batched form: nsteps consecutive MD steps step0..step0+nsteps-1
 * of n walkers with their own grids in one launch, equal per step and walker
 * to abp_step followed by abp_forces. Coordinates of step t at record
 * coord_offsets_dev[w] + t * coord_step_stride + i; forces written (by mode)
 * at force_offsets_dev[w] + t * force_step_stride + i. Walkers that share a
 * grid are rejected (use abp_step). */
abp_status abp_run(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                   const int64_t *coord_offsets_dev, int64_t coord_step_stride, void *forces_dev,
                   const int64_t *force_offsets_dev, int64_t force_step_stride, int mode, int64_t step0, int nsteps);

/* The plain one-walker-per-launch form of abp_step + abp_forces: for every
 * walker, separate CV, deposit and interpolation/force kernel launches from a
 * host loop (the comparison point for the batched form). Same arguments and
 * results as one step of abp_run. */
abp_status abp_step_plain(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev,
                          int coords_dtype, const int64_t *coord_offsets_dev, void *forces_dev,
                          const int64_t *force_offsets_dev, int mode, int64_t step);

/* ---- closed-loop dynamics ------------------------------------------------------- */

/* A model MD engine around the force call, on the device: the paper's bias
 * routine sits inside the biased MD cycle (Figure "cycle": coordinates in,
 * bias force out, added to the MD force), so the coordinates of step t + 1
 * depend on the bias force of step t. abp_md_run closes that loop without
 * leaving the GPU. Every CV atom moves by overdamped Langevin dynamics
 *   x <- x + dt mu F + sqrt(2 mu kT dt) xi,
 *   F  = F_bias - sum_k dU/ds_k ds_k/dx,
 * F_bias the step's bias force (steps a1..a5, as abp_run computes it) and U
 * an optional potential of the walker's CVs; xi three standard normals per
 * atom and step: Philox-4x32-10 (Salmon et al., "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11) of the counter (atom index, step low 32 bits,
 * step high 32 bits, the walker's stream) under the key (seed low 32 bits,
 * seed high 32 bits); each output word's top 24 bits give u = (j + 1/2) 2^-24,
 * and Box-Muller gives n0 = r0 cos(2 pi u1), n1 = r0 sin(2 pi u1),
 * n2 = r2 cos(2 pi u3), r = sqrt(-2 ln u). The paper has no counterpart (its
 * MD engine is GROMACS). */
#define ABP_POT_NONE 0
#define ABP_POT_DOUBLE_WELL 1  /* U = dw_a (s_0^2 - dw_b^2)^2 */
#define ABP_POT_MULLER_BROWN 2 /* U = mb_scale sum_{i<4} mb_A[i] exp(mb_a[i] X'^2 + mb_b[i] X' Y' + mb_c[i] Y'^2),
                                  X' = X - mb_x0[i], Y' = Y - mb_y0[i], X = mb_map[0] s_0 + mb_map[1],
                                  Y = mb_map[2] s_1 + mb_map[3] (the surface of Mueller and Brown,
                                  Theor. Chim. Acta 53 (1979), on an affine image of the CV box) */

typedef struct {
  double dt;        /* time step (ps) */
  double mobility;  /* mu (nm^2 / (kJ/mol ps)) */
  double kT;        /* thermal energy of the noise (kJ/mol) */
  uint64_t seed;    /* Philox key */
  int potential;    /* ABP_POT_* */
  double dw_a, dw_b;
  double mb_scale;
  double mb_map[4];
  double mb_A[4], mb_a[4], mb_b[4], mb_c[4], mb_x0[4], mb_y0[4];
} abp_md_desc;

/* nsteps closed-loop MD steps step0..step0+nsteps-1 of n walkers in one
 * launch. coords_dev holds each walker's atoms at step0 (records at
 * coord_offsets_dev[w] + i, dtype as for abp_run) and receives them after
 * the last step's move (in place). streams (host, n values) are the walkers'
 * noise streams. Optional outputs (NULL to skip): traj_dev, the coordinates
 * each step's bias was evaluated at (records at traj_offsets_dev[w] +
 * t * traj_step_stride + i); forces_dev, each step's bias force (records at
 * force_offsets_dev[w] + t * force_step_stride + i, by mode; without it
 * abp_forces delivers the last step's). Walkers whose CVs are COM
 * distances, dihedrals or RMSDs run one warp each (steps chained on the
 * device); walkers of the phased form (a shared grid or a large walker) run
 * their step's launches followed by the move, and take ABP_POT_NONE only.
 * Other walkers (a coordination number in the fused form) are rejected with
 * ABP_ERR_UNSUPPORTED. A walker that meets non-finite coordinates stops
 * there (its state reports ABP_WFLAG_NONFINITE; abp_sync returns
 * ABP_ERR_NONFINITE). Asynchronous on the context stream. */
abp_status abp_md_run(abp_ctx *ctx, abp_walker *const *walkers, int n, void *coords_dev, int coords_dtype,
                      const int64_t *coord_offsets_dev, const abp_md_desc *md, const uint32_t *streams,
                      void *traj_dev, const int64_t *traj_offsets_dev, int64_t traj_step_stride, void *forces_dev,
                      const int64_t *force_offsets_dev, int64_t force_step_stride, int mode, int64_t step0,
                      int nsteps);

/* ---- readouts ------------------------------------------------------------ */

/* Copies the grid's fields, [nodes][1 + ncv] (V then dV/dxi_k), to dst as
 * ABP_F32 or ABP_F64 (FP32_COMP grids return sum + compensation). Syncs. */
abp_status abp_bias_readout(abp_ctx *ctx, const abp_grid *grid, void *dst, int dst_is_device, int dtype);
/* Replaces the grid's fields by src ([nodes][1 + ncv], ABP_F32 or ABP_F64);
 * an FP64 source is split exactly into value + compensation on FP32_COMP
 * grids. Syncs. */
abp_status abp_bias_upload(abp_ctx *ctx, abp_grid *grid, const void *src, int src_is_device, int dtype);

/* Checkpoint and restart (not a paper operation: the bias is state a long
 * run saves and reloads). abp_grid_save copies the grid's node records as
 * stored (value and compensation words of FP32_COMP grids, then for a grid
 * created with shared = 1 its FP64 accumulator shadow), abp_grid_record_bytes
 * of them, to dst; abp_grid_restore writes such bytes back into a grid of
 * the same description. A walker whose grid is restored resumes its run bit
 * for bit (abp_bias_readout / abp_bias_upload go through FP64 values and
 * agree only to rounding). Both sync. */
size_t abp_grid_record_bytes(const abp_grid *grid);
abp_status abp_grid_save(abp_ctx *ctx, const abp_grid *grid, void *dst, int dst_is_device);
abp_status abp_grid_restore(abp_ctx *ctx, abp_grid *grid, const void *src, int src_is_device);
/* s_t[3], V_b(s_t), dV_b/ds[3] and flags of the walker's last step. Syncs.
 * Returns ABP_ERR_NONFINITE if that step saw non-finite coordinates. */
abp_status abp_walker_readout(abp_ctx *ctx, const abp_walker *walker, double *s, double *V, double *dV,
                              int *flags);

/* Deposit log: when enabled with a capacity, every deposit appends one
 * abp_deposit_rec (records beyond the capacity are counted, not stored).
 * Readout syncs and returns the stored records in device order per call. */
abp_status abp_deposit_log_enable(abp_ctx *ctx, size_t capacity);
abp_status abp_deposit_log_readout(abp_ctx *ctx, abp_deposit_rec *dst, size_t cap, size_t *n_out,
                                   size_t *n_total);
abp_status abp_deposit_log_clear(abp_ctx *ctx);

/* ---- shared grids across GPUs: hill exchange -------------------------------- */

/* Walkers of one multiple-walker run may live on several GPUs, each GPU
 * holding a replica of the shared grid. A step then runs in three calls:
 * abp_shared_hills (CVs and heights, from this replica, no deposit), an
 * exchange of the hill records among the GPUs (by the caller, e.g. an
 * all-gather), abp_grid_apply_hills with every record of the step in
 * (rank, walker) order on every replica, and abp_shared_forces. Replicas that
 * start equal and apply the same records stay bit-identical. The paper's
 * counterpart is the master rank that gathers CV atoms and returns forces
 * (SI "Minimization of Interprocess Communications"); here only the few bytes
 * of each hill move. */
typedef struct {
  double s[3];        /* hill centre s_t */
  double height;      /* h */
  int64_t step;
  int32_t walker_id;
  int32_t pad;
} abp_hill;

/* Steps a1 + a2 of MD step `step` for walkers on one shared grid (created
 * with shared = 1): writes to host memory, in list order, the hills the
 * walkers deposit this step (none if step % stride != 0), without depositing
 * them; *n_out receives the count. Syncs. */
abp_status abp_shared_hills(abp_ctx *ctx, abp_walker *const *walkers, int n, const void *coords_dev, int coords_dtype,
                            const int64_t *coord_offsets_dev, int64_t step, abp_hill *hills_out, size_t cap,
                            size_t *n_out);
/* Deposits n hill records (host memory) into the shared grid of `shape_walker`,
 * whose sigma and cutoff every record uses, exactly as if they were applied one
 * after another in list order: records whose stencil boxes cannot overlap go
 * in one launch, overlapping ones in list order, without atomics. */
abp_status abp_grid_apply_hills(abp_ctx *ctx, const abp_walker *shape_walker, const abp_hill *hills, size_t n);
/* Steps a4 + a5 after the step's hills are applied: forces for the walkers of
 * the last abp_shared_hills call, written as abp_run writes them. */
abp_status abp_shared_forces(abp_ctx *ctx, abp_walker *const *walkers, int n, void *forces_dev, int forces_dtype,
                             const int64_t *force_offsets_dev, int mode, int64_t step);

/* ---- serving: continuous batching of step requests ------------------------ */

/* A request loop over many concurrent simulations (one walker each): every
 * simulation's grid and state stay on the device; callers submit one MD step
 * at a time (host coordinates in, host forces out) from any thread; a
 * launcher thread packs the requests that are ready into the next launch of
 * the fused kernel on one of nstreams streams while earlier launches are
 * still in flight (continuous batching), and a delivery thread hands each
 * finished request back through abp_server_poll. A simulation's steps run
 * in order (each depends on the
 * grid after the previous one): a launch takes at most one request of a
 * simulation, and when the simulation's previous request is still running
 * in another launch, the new launch's kernel waits on the device for that
 * one's kernel, so the host can pack the next launch meanwhile. Results
 * come back in launch order, so one simulation's results arrive in step
 * order. A walker's result is the same alone and in any mix of requests.
 * A launch uploads its requests' coordinates and its walker table in one
 * host-to-device copy. When it runs out of work the launcher thread spins
 * for up to 50 us before it sleeps, so that a request arriving then is taken
 * without a thread wake-up (one host core is busy during that spin).
 * The server owns the context's stream while it runs. */
typedef struct abp_server abp_server;

typedef struct {
  int max_batch;   /* requests per launch (0 = 4096) */
  int max_atoms;   /* largest walker block accepted (0 = 1024 atoms) */
  int nstreams;    /* launches in flight at once (0 = 2) */
} abp_server_desc;

typedef struct {
  int64_t sim;        /* simulation id */
  int64_t step;       /* MD step of the request */
  uint64_t tag;       /* the caller's tag */
  double t_submit;    /* host steady-clock seconds at submit */
  double t_done;      /* host steady-clock seconds when the forces were in forces_host */
  int32_t status;     /* ABP_OK, or an error code (then forces_host is untouched) */
  int32_t batch;      /* requests in the launch that served it */
} abp_result;

abp_status abp_server_create(abp_ctx *ctx, const abp_server_desc *desc, abp_server **out);
/* Stops the worker after the requests in flight finish; unfinished queued
 * requests are dropped. Frees every admitted simulation. */
void abp_server_destroy(abp_server *srv);
/* Admits a simulation: creates its grid and walker against the context's
 * HBM budget; returns ABP_ERR_ADMISSION (nothing allocated) when they do not
 * fit, so the caller can retry after abp_server_release frees memory.
 * Simulations sharing a grid are not served (walkers on own grids only). */
abp_status abp_server_admit(abp_server *srv, const abp_grid_desc *grid, const abp_walker_desc *walker,
                            int64_t *sim);
/* Releases a simulation once its requests have finished (waits for them). */
abp_status abp_server_release(abp_server *srv, int64_t sim);
/* Copies a simulation's bias grid (as abp_bias_readout) once its queued and
 * running requests have finished (waits for them, up to 60 s, then
 * ABP_ERR_TIMEOUT): the free-energy estimate of a served simulation. */
abp_status abp_server_bias_readout(abp_server *srv, int64_t sim, void *dst, int dst_is_device, int dtype);
/* Queues MD step `step` of simulation `sim`: coords_host (natoms float
 * records x, y, z, pad) is copied before the call returns; the bias forces
 * are written (overwrite) to forces_host (natoms float records, caller-owned,
 * valid until the request is polled). */
abp_status abp_server_submit(abp_server *srv, int64_t sim, int64_t step, const float *coords_host,
                             float *forces_host, uint64_t tag);
/* n requests in one call: request k is (sims[k], steps[k], tags[k]); its
 * coordinates follow those of request k-1 in coords_host (natoms records of
 * its simulation each, copied before the call returns) and its forces land
 * at the same offset of forces_host. They are queued in order, in chunks of
 * 2048, so that the first launches start while later chunks are copied; all
 * carry the call's time as t_submit. Unknown simulations or negative steps
 * are rejected before anything is queued; a simulation released by another
 * thread during the call ends it with ABP_ERR_INVALID_ARG after the chunks
 * before it were queued. */
abp_status abp_server_submit_many(abp_server *srv, int n, const int64_t *sims, const int64_t *steps,
                                  const float *coords_host, float *forces_host, const uint64_t *tags);
/* Cancels the requests of simulation `sim` that are still queued (not yet
 * packed into a launch): each comes back through abp_server_poll with status
 * ABP_ERR_CANCELLED and its forces_host untouched; requests already launched
 * finish normally. *n_cancelled (may be NULL) receives how many were
 * cancelled. The simulation stays admitted; later submits are served. */
abp_status abp_server_cancel(abp_server *srv, int64_t sim, int64_t *n_cancelled);
/* Up to cap finished requests, oldest first; waits up to wait_ms for the
 * first one when none is ready (0 = do not wait). */
abp_status abp_server_poll(abp_server *srv, abp_result *out, int cap, int *n_out, int wait_ms);
/* Counters: requests submitted, finished, launches, and requests queued now. */
abp_status abp_server_stats(abp_server *srv, int64_t *submitted, int64_t *finished, int64_t *launches,
                            int64_t *queued);
/* Seconds the server's two threads have spent, since the server was
 * created, in each phase: the launcher filling slots from the ready
 * simulations (under the server lock) and packing and launching them (host
 * copies into pinned memory, asynchronous copies and the kernel launch); the
 * deliverer waiting for launched slots to finish on the GPU and delivering
 * them (forces into the callers' buffers, results queued). Any pointer may
 * be NULL. */
abp_status abp_server_times(abp_server *srv, double *fill_s, double *launch_s, double *complete_s, double *wait_s);
/* Host steady-clock seconds (the clock of abp_result). */
double abp_server_now(void);

/* ---- checked build -------------------------------------------------------- */

/* The library compiled with -DABP_CHECKED (paper_1609_09833_gb300.build,
 * checked=True) checks every grid node index its kernels read or write:
 * an index outside its grid is counted here and replaced by node 0, so the
 * access stays inside the grid's allocation (the substitute for a device
 * memory checker). Waits for the context stream, then returns the count
 * since the context was created in *count and whether this library is the
 * checked build in *checked (the normal build always counts 0). Either
 * pointer may be NULL. */
abp_status abp_checked_violations(abp_ctx *ctx, uint64_t *count, int *checked);

/* ---- allocation-free step -------------------------------------------------- */

/* abp_step_static: one MD step (a1..a5) of one walker, allocating nothing on
 * the device. The paper has no counterpart. It serves callers for which a
 * cudaMalloc or cudaFree inside the step is not acceptable:
 *   - a plugin inside a host MD engine that hands out GPU memory from its own
 *     pool with a fixed budget: an allocation made around that pool can fail
 *     once the engine has taken the card's memory, and the engine cannot see
 *     or account for it;
 *   - a step loop that keeps several streams busy: cudaFree synchronises the
 *     whole device, so an allocating bias call would stall the engine's other
 *     work every time it released scratch;
 *   - a long run under a per-process memory limit, where the bias must not be
 *     able to fail for want of memory hours into the run.
 * It runs the kernels of abp_step_plain and gives the same results, but keeps
 * everything beyond the caller's buffers (the walker description, its atom
 * lists, the Jacobian passed between the kernels, a counter) in one static
 * device array of ABP_STATIC_SCRATCH_BYTES. The CUDA runtime reserves that
 * array when it loads the library's module on a device (with lazy module
 * loading: at the first use of one of the library's kernels or symbols there,
 * which may be this call's first invocation) and holds it until the process
 * exits; the call itself makes no cudaMalloc, cudaFree or other allocating
 * call.
 *
 *   device, cuda_stream   the GPU and the cudaStream_t to run on (the caller's
 *                         current device is restored on return)
 *   grid_desc             the grid (as for abp_create_grid)
 *   grid_records_dev      caller-owned grid storage: nodes records of 16 bytes
 *                         (ncv = 1) or 32 bytes (ncv > 1), node order and
 *                         record layout of the library's grids (FP32_COMP:
 *                         float {V, dV0, cV, cdV0} or float {V, dV0, dV1, dV2},
 *                         {cV, cdV0, cdV1, cdV2}, c = compensation; FP64:
 *                         double {V, dV0} or {V, dV0, dV1, dV2}); zero it
 *                         before the first step (V_b = 0); updated in place
 *   walker_desc           the walker (as for abp_walker_create; host arrays);
 *                         COM distance, dihedral and coordination-number CVs
 *                         (an RMSD CV returns ABP_ERR_UNSUPPORTED)
 *   coords_dev, forces_dev  the walker's atoms and its force records
 *   mode, step            as for abp_step_plain
 *
 * Every call shares the array and leaves the last call's contents in it; the
 * call copies what the kernels read into it (one cudaMemcpyAsync on
 * cuda_stream from a host staging image that the call owns) before they run,
 * so calls must not overlap on the GPU: two calls in flight at once (other
 * streams, other host threads) race on the array. The call is asynchronous on
 * cuda_stream; it reports no non-finite coordinates (forces are zeroed,
 * nothing is deposited). A walker whose description, lists and Jacobian need
 * more than ABP_STATIC_SCRATCH_BYTES is rejected with ABP_ERR_INVALID_ARG. */
#define ABP_STATIC_SCRATCH_BYTES (1u << 20)
abp_status abp_step_static(int device, void *cuda_stream, const abp_grid_desc *grid_desc, void *grid_records_dev,
                           const abp_walker_desc *walker_desc, const void *coords_dev, int coords_dtype,
                           void *forces_dev, int mode, int64_t step);

/* ---- measurement ------------------------------------------------------------ */

/* The device's FP32 FMA throughput (the paper has no counterpart: it is the
 * denominator of the arithmetic rooflines of the coordination-number pair
 * loops): one launch of 8 x (multiprocessors) CTAs of 256 threads, each
 * thread advancing 8 independent FMA chains for `iters` rounds (2 flops per
 * FMA), timed with CUDA events on cuda_stream after a short warm-up launch.
 * Writes FLOP/s to *flops_per_s and the timed seconds to *seconds (may be
 * NULL). Allocates and frees a small output buffer; restores the caller's
 * current device; synchronous. */
abp_status abp_fp32_fma_peak(int device, void *cuda_stream, int iters, double *flops_per_s, double *seconds);

/* Waits for the context stream; returns ABP_ERR_NONFINITE if any walker
 * stepped since the last sync saw non-finite coordinates. */
abp_status abp_sync(abp_ctx *ctx);
const char *abp_last_error(void);
/* Library version string. */
const char *abp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ABP_H */
