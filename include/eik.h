/*
 * eik.h -- C ABI of the GB300 (sm_103a) Eikonal solver libeik.so.
 *
 * The library solves the first-order upwind (Godunov) discretization of the
 * static Eikonal equation |grad u(x)| F(x) = 1 with u = q on an exit set
 * (Chacon & Vladimirsky, "A parallel Heap-Cell Method for Eikonal
 * equations", arXiv:1306.4743, Sec. 1.1, Eq. 2) on a uniform 3D grid, by a
 * GPU restatement of the parallel Heap-Cell Method (Sec. 4-5, Alg. 1-3):
 * the grid is split into cells of n^3 nodes, each cell is swept with the
 * modified Locking Sweeping update of Alg. 2 in alternating directions,
 * cells whose border values changed are flagged, and a persistent kernel
 * takes the next cells from a device-side bucketed queue keyed on the cell
 * value of Eq. 3.
 *
 * Grid convention (Sec. 1.1): node (i,j,k), 0 <= i < nx, 0 <= j < ny,
 * 0 <= k < nz, sits at (i h, j h, k h); every array below holds one entry
 * per node at linear index i + nx*(j + ny*k) (i fastest).  Values outside
 * the grid are +infinity (Sec. 1.1); exit nodes (the set Q' of Sec. 4) keep
 * u = q exactly.
 *
 * Ownership: the caller owns every input and output buffer; the library
 * copies what it needs during a call and keeps no caller pointer after the
 * call returns (for eik_submit: after eik_poll reports completion).  The
 * library owns an eik_ctx and all device memory inside it.
 *
 * Errors: every entry point returns an eik_status code; nothing aborts the
 * process.  A device wait that exceeds opts.spin_cap_us, or a device fault,
 * surfaces as EIK_ETIMEOUT / EIK_ECUDA.  eik_strerror() names each code.
 *
 * Threads: one eik_ctx may be used by one host thread at a time.
 */
#ifndef EIK_H
#define EIK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque solver context (owned by the library). */
typedef struct eik_ctx eik_ctx;

/* Status codes. */
enum {
  EIK_OK = 0,
  EIK_EINVAL = 1,     /* bad argument: dims < 1, h <= 0, F <= 0 or not finite,
                         no exit node, q not finite, tol < 0 or NaN */
  EIK_ENOMEM = 2,     /* device or host allocation failed */
  EIK_EBUDGET = 3,    /* the solve needs more device memory than
                         opts.hbm_budget_bytes allows */
  EIK_ECUDA = 4,      /* a CUDA call failed */
  EIK_ETIMEOUT = 5,   /* a device wait passed opts.spin_cap_us without progress */
  EIK_ENOCONV = 6,    /* a cell passed the sweep limit of one visit */
  EIK_ECANCELLED = 7, /* a submitted request was cancelled */
  EIK_EQUEUE = 8,     /* internal device queue inconsistency */
  EIK_ENOTFOUND = 9   /* unknown ticket */
};

/* Arithmetic of the sweeps. */
typedef enum {
  EIK_FP64 = 0,        /* every sweep in double precision */
  EIK_FP32_POLISH = 1  /* bulk sweeps in single precision, then double
                          precision polishing sweeps from the single-precision
                          result (Sec. 6.4 studies the single-precision
                          behaviour; the polish restores double precision) */
} eik_precision;

/* Options of a context.  Fill with eik_opts_default() and change fields. */
typedef struct {
  int device;               /* CUDA device ordinal (default 0) */
  int precision;            /* eik_precision (default EIK_FP32_POLISH) */
  int cell_n;               /* nodes per cell side: 4, 8 or 16; 0 = choose by
                               grid size: 16 from 2^21 nodes up, else 8
                               (default 0) */
  int max_ctas;             /* CTAs of the persistent cell kernel; 0 = every
                               CTA that fits on the device at once (default) */
  size_t hbm_budget_bytes;  /* device-memory limit of this context; 0 = none */
  uint64_t spin_cap_us;     /* longest device wait without global progress,
                               in microseconds (default 5,000,000); 0 makes
                               every idle wait fail at once (test hook) */
  double bucket_width;      /* width of one queue bucket in units of
                               (cell edge x front slowness), the front
                               slowness being the harmonic mean of s = h / F,
                               h / mean(F); <= 0 = default 0.25 */
  int max_sweeps_per_visit; /* sweep limit of one cell visit (default 4096) */
  int queue_order;          /* 0 = strict: the next bucket starts once every
                               cell of the current one is finished;
                               1 = relaxed: once the current bucket is empty
                               (default) */
  double bulk_kappa_rel;    /* EIK_FP32_POLISH only: change threshold of the
                               FP32 bulk sweeps, in units of (cell edge x front
                               slowness).  Stopping the bulk early leaves
                               values high, never low, and the FP64 polish
                               starts above the fixed point, so this trades
                               bulk sweeps for polish sweeps and does not
                               change the result.  0 (default) = chosen per
                               solve from the dispersion of s = h / F over the
                               launch, r = mean(s) mean(1 / s): 3e-3 r^2, at
                               most 1 (fine where s is nearly uniform, coarse
                               where it spreads widely and fronts revisit
                               cells along faster detours). */
  int use_graphs;           /* eik_solve_batch_device: capture the launch
                               sequence as a CUDA graph and replay it while
                               the arguments repeat (default 1) */
  int cell_key;             /* cell value a flag gives the neighbour cell:
                               0 = Eq. 3, the smallest flagging border value
                               (default); 1 = Eq. 4, the largest one plus
                               (n + 1) h / 2 over the speed at the neighbour's
                               centre, with cell values kept (not reset to
                               +inf) when a cell is taken (Sec. 6.8) */
  int warps_per_cell;       /* warps that sweep one 16^3 cell together: 4, 6
                               or 8 (6: one thread per node of the largest
                               plane; 8: one thread per (j, k) pencil); 0 =
                               the autotuned value, else 8 for the FP32 bulk
                               and 6 for FP64 sweeps */
  uint64_t serve_batch_nodes; /* serving: a batch takes waiting requests until
                                 it holds this many grid nodes (at least one
                                 request); 0 = default 64 M.  Smaller batches
                                 start sooner, larger ones use the device
                                 better. */
  double polish_lift;       /* EIK_FP32_POLISH only: the FP32 result is raised
                               by this fraction of itself before the monotone
                               FP64 polish, so that the polish starts above the
                               fixed point (FP32 rounding grows ~2^-24 u per
                               node along a characteristic); 0 = default 2^-11.
                               A negative value starts below the fixed point,
                               where monotone sweeps cannot arrive: the
                               residual check then sends every cell to the
                               replace-mode polish (fallback_used = 1), which
                               is how that path is tested. */
} eik_opts;

/* Counters and results of one solve (of the whole batch for batch calls). */
typedef struct {
  double seconds;               /* device time from the first init kernel to
                                   the final u on the device */
  uint64_t cell_visits;         /* cells taken from the queue, bulk pass */
  uint64_t sweeps;              /* directional sweeps, bulk pass */
  uint64_t node_updates;        /* local solves, bulk pass */
  uint64_t polish_visits;       /* cells taken from the queue, FP64 polish */
  uint64_t polish_sweeps;
  uint64_t polish_node_updates;
  uint64_t queue_pushes;        /* bucket insertions, both passes */
  uint64_t nonfinite;           /* nodes left non-finite (0 on success) */
  uint64_t nodes;               /* nx*ny*nz summed over instances */
  int cell_n_used;
  int precision_used;
  double residual_max;          /* max |u - Lambda(u)| over non-exit nodes,
                                   recomputed in FP64 after the solve */
  double u_max;                 /* largest finite u */
  double seconds_bulk;          /* device time of the bulk cell kernel */
  double seconds_polish;        /* device time of the polish cell kernel */
  uint64_t kernel_launches;     /* CUDA kernels this call launched */
  int grid_ctas;                /* CTAs of the persistent cell kernel */
  int fallback_used;            /* 1 if the replace-mode polish ran */
  double busy_seconds_bulk;     /* sum over cell visits of their duration */
  double busy_seconds_polish;
  uint64_t fallback_visits;
  double phase_seconds[2][4];   /* [bulk, polish] x [waiting in the queue pop,
                                   TMA staging, sweeps, write-back + flags + retire],
                                   summed over workers */
  uint64_t revisits[2];         /* [bulk, polish]: visits of a cell that had
                                   converged before (restarted at its flagged faces) */
  uint64_t revisit_sweeps[2];   /* ... the sweeps of those visits */
  uint64_t revisit_updates[2];  /* ... and their node updates */
  uint64_t max_visit_sweeps[3]; /* [bulk, polish, fallback]: most sweeps in one visit */
  double seconds_stage[3];      /* device time of the streaming stages: [init
                                   (inputs to queued exit cells), FP32 -> FP64
                                   hand-over and polish schedule, residual check +
                                   fallback + copy-out] */
  int warps_per_cell_used;      /* warps per 16^3 cell of the bulk sweeps */
  int reserved_stats;
  double bulk_kappa;            /* EIK_FP32_POLISH: the change threshold the
                                   bulk sweeps used (absolute); 0 for EIK_FP64 */
} eik_stats;

/* Default options. */
int eik_opts_default(eik_opts *opts);

/* Create a context on opts->device (NULL opts = defaults).  *out is set to a
 * new context on success and to NULL on failure. */
int eik_create(eik_ctx **out, const eik_opts *opts);

/* Free a context and its device memory.  NULL is accepted. */
int eik_destroy(eik_ctx *ctx);

/* Static English text for a status code. */
const char *eik_strerror(int status);

/* sizeof(eik_opts) and sizeof(eik_stats) as compiled into the library, so
 * that a binding can check its own copies of the two structs.  Either
 * pointer may be NULL.  Always returns EIK_OK; needs no device. */
int eik_struct_sizes(size_t *opts_bytes, size_t *stats_bytes);

/*
 * Solve one grid (Eq. 2), host buffers.
 *   dims[3]  = {nx, ny, nz}, each >= 1
 *   h        = grid step, > 0
 *   F        = speed per node (nx*ny*nz floats), > 0 and finite off the exit set
 *   src_mask = exit set Q' (nx*ny*nz bytes), nonzero = exit node; at least one
 *   q        = exit values (nx*ny*nz doubles), read only where src_mask != 0,
 *              finite
 *   tol      = kappa of the early-termination rule of Sec. 6.3: a local
 *              update that changes a value by no more than tol does not count
 *              as a change, neither for stopping a cell's sweeps nor for
 *              flagging a neighbouring cell (tol = 0: sweep until no value
 *              changes).  Applies to the FP64 sweeps of either precision mode.
 *   u_out    = caller-owned nx*ny*nz doubles, written on EIK_OK
 *   stats    = may be NULL
 * Host buffers that are page-locked (cudaHostAlloc / cudaHostRegister) are
 * used in place: the device reads F and q (q only at exit nodes) and writes
 * u_out over the CPU-GPU link instead of the call copying them; pageable
 * buffers are copied.  Either way the call returns with u_out written.
 * Returns EIK_OK or an error code; on error u_out is unspecified.
 */
int eik_solve(eik_ctx *ctx, const int64_t dims[3], double h, const float *F,
              const uint8_t *src_mask, const double *q, double tol,
              double *u_out, eik_stats *stats);

/*
 * Same as eik_solve with every array in device memory of ctx's device.
 * The work runs on `stream` (a cudaStream_t; NULL = the legacy default
 * stream) and the call returns after the stream has finished it.
 */
int eik_solve_device(eik_ctx *ctx, const int64_t dims[3], double h,
                     const float *F_dev, const uint8_t *src_mask_dev,
                     const double *q_dev, double tol, double *u_out_dev,
                     void *stream, eik_stats *stats);

/*
 * Autotuner.  Times the solve of a representative grid (host buffers, as
 * eik_solve) for each worker shape -- cells of 4^3 and 8^3 (one warp per
 * cell; 4^3 only up to 2^22 nodes) and 16^3 cells with the default shapes
 * (8 warps for the FP32 bulk, 6 for FP64 sweeps) or 4, 6 or 8 warps in every
 * pass -- with one or two cell-kernel CTAs per SM, keeps the fastest for this
 * context, and uses it for later solves whose size falls in the same
 * power-of-two bucket of node count while opts.cell_n, opts.max_ctas and
 * opts.warps_per_cell are 0.  Returns the cell size and CTA count in
 * *best_n / *best_ctas (either may be NULL); the warps per cell show in
 * eik_stats.warps_per_cell_used of later solves.  Cell size 32 is not
 * offered: a 32^3 cell with its halo does not fit shared memory next to its
 * slowness.
 */
int eik_autotune(eik_ctx *ctx, const int64_t dims[3], double h, const float *F,
                 const uint8_t *src_mask, const double *q, double tol, int *best_n,
                 int *best_ctas);

/*
 * Solve `count` independent grids in one persistent launch (host buffers).
 * Instance t uses dims[3t..3t+2], h[t], F[t], src_mask[t], q[t], u_out[t].
 * Cells of all instances share one device queue.  stats (may be NULL) sums
 * over the batch.
 */
int eik_solve_batch(eik_ctx *ctx, int count, const int64_t *dims,
                    const double *h, const float *const *F,
                    const uint8_t *const *src_mask, const double *const *q,
                    double tol, double *const *u_out, eik_stats *stats);

/* Device-buffer variant of eik_solve_batch (all arrays in device memory;
 * the pointer tables themselves are host arrays).  With opts.use_graphs the
 * first call with a given set of arguments runs plainly and then captures
 * the whole launch sequence (copies of the small tables, init kernels, the
 * persistent cell kernels, residual, read-back) as one CUDA graph; later
 * calls with the same grids, buffers, tolerance and stream replay it. */
int eik_solve_batch_device(eik_ctx *ctx, int count, const int64_t *dims,
                           const double *h, const float *const *F_dev,
                           const uint8_t *const *src_mask_dev,
                           const double *const *q_dev, double tol,
                           double *const *u_out_dev, void *stream,
                           eik_stats *stats);

/*
 * Serving (continuous batching).  eik_submit queues one solve (host buffers,
 * same arguments as eik_solve) and returns a ticket at once.  The library
 * reads F, src_mask and q, and writes u_out, asynchronously: the caller keeps
 * all four buffers alive and unchanged until eik_poll reports the ticket
 * done or eik_cancel succeeds.  Requests are admitted to the device in
 * arrival order, in batches, on a few concurrent execution slots, while the
 * memory of the batches on the device fits opts.hbm_budget_bytes; requests
 * that arrive while others run start as soon as a slot and memory free up.
 * A request that alone exceeds the budget completes with EIK_EBUDGET.
 * eik_poll advances the queue (retires finished batches, admits waiting
 * requests) and sets *done = 1 once the ticket's u_out is written; it then
 * returns the ticket's status, and the ticket is forgotten.  eik_cancel
 * drops a ticket that has not completed; a batch already on the device
 * finishes into a private buffer, except that a page-locked u_out
 * (cudaHostAlloc / cudaHostRegister) is written in place by the device, so
 * eik_cancel of such a request on the device first waits for its batch to
 * finish.  Page-locked F and q are read in place (no copy), as in
 * eik_solve.  Unknown tickets give EIK_ENOTFOUND.
 */
int eik_submit(eik_ctx *ctx, const int64_t dims[3], double h, const float *F,
               const uint8_t *src_mask, const double *q, double tol,
               double *u_out, uint64_t *ticket);
int eik_poll(eik_ctx *ctx, uint64_t ticket, int *done, eik_stats *stats);
int eik_cancel(eik_ctx *ctx, uint64_t ticket);

/*
 * Allocation-free FP64 solve (this entry point has no counterpart in the
 * paper; it exists for the callers below).
 *
 * Some callers cannot allocate device memory while they solve: programs
 * whose own caching allocator has reserved the device memory up front (a
 * cudaMalloc would fail, or force that allocator to give memory back),
 * latency-critical loops where an allocation can stall behind a device-wide
 * synchronisation, and plug-in code whose host framework only lets it use
 * memory it was handed.  eik_solve_device_noalloc needs no context and calls
 * no allocating routine: its working memory is one fixed device array of
 * EIK_NOALLOC_SCRATCH_BYTES inside the library, which every device that
 * loads the library holds until the process exits.
 *
 * Arguments as eik_solve_device (device buffers on the current device,
 * stream = cudaStream_t or NULL); the sweeps run in FP64 with cells of 8^3
 * nodes.  The call enqueues the solve on `stream`, waits for that stream to
 * finish it and then returns; stats (may be NULL) gets the counters and the
 * residual, not the timings.
 *
 * Limits and sharing:
 *  - a grid needs about 17 bytes of scratch per node plus padding; larger
 *    grids (above roughly 150^3 nodes for a cube, and any grid above
 *    EIK_NOALLOC_SCRATCH_BYTES / 16 nodes) are rejected with EIK_EBUDGET
 *    before any device work;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture;
 *  - all calls share the one array (per device), and the array keeps the
 *    last call's contents; a call initialises everything it reads, but two
 *    calls whose device work overlaps (different streams, or host threads)
 *    race on the array and give wrong results.  Calls from several host
 *    threads are serialised on the host.
 */
#define EIK_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int eik_solve_device_noalloc(const int64_t dims[3], double h, const float *F_dev,
                             const uint8_t *src_mask_dev, const double *q_dev,
                             double tol, double *u_out_dev, void *stream,
                             eik_stats *stats);

/*
 * Whole-grid sweeping baseline (the paper's parallel comparator DFSM,
 * Sec. 2-3 and Tables 4-6): Fast Sweeping of the whole grid in the 8
 * directions of the standard order, each direction over the planes
 * i + j + k = C of that direction with the nodes of a plane updated in
 * parallel, in FP64, until a sweep lowers no value by more than tol (tol = 0:
 * until no value changes).  Same problem and arguments as eik_solve_device
 * (device pointers, layout (nz, ny, nx), i fastest; u_out_dev caller-owned),
 * plus max_sweeps (1 .. 2^20).  On success *sweeps (nullable) is the number
 * of sweeps, and changed_per_sweep / max_drop_per_sweep (host arrays of
 * max_sweeps entries, nullable) the count of values lowered by more than
 * tol in each sweep and the largest such decrease.  Allocates its working
 * memory (~16 B per node) for the call and frees it; runs on the current
 * device and stream and synchronises the stream.  EIK_EINVAL for bad
 * arguments, F <= 0 or non-finite, non-finite q, or no exit node;
 * EIK_ENOMEM; EIK_ENOCONV when the last allowed sweep still changed a
 * value (u_out holds that iterate); EIK_ETIMEOUT if a device-wide barrier
 * waits longer than 5 s; EIK_ECUDA.
 */
int eik_dfsm_solve_device(const int64_t dims[3], double h, const float *F_dev,
                          const uint8_t *src_mask_dev, const double *q_dev, double tol,
                          int64_t max_sweeps, double *u_out_dev, void *stream,
                          int64_t *sweeps, int64_t *changed_per_sweep,
                          double *max_drop_per_sweep, eik_stats *stats);

/*
 * Diagnostic: accuracy of the device local solve of Eq. 2 (Sec. 1.1) used
 * by the FP64 sweeps, against the direct FP64 evaluation of the same root
 * (shifted closed forms with an FP64 square root, the form the residual
 * certificate uses), on `count` inputs drawn on the device from a
 * counter-based generator keyed by `seed`: s = h / F with h log-uniform in
 * [2^-10, 2^-4] and F uniform in [0.05, 2], neighbour values a base uniform
 * in [0, 2) plus offsets uniform in [0, 2s] (one in eight +inf), so that the
 * one-, two- and three-term cases all occur.  On success *max_ulps is the
 * largest difference in units in the last place of the direct result and
 * *max_rel the largest difference in units of (one ulp of the direct
 * result + 2^-44 s), the accuracy the sweeps' solve is built for.  Runs on `device`, allocates
 * and frees a few bytes of device memory, synchronises the device.
 * Returns EIK_EINVAL for count < 1 or NULL outputs, EIK_ECUDA on a CUDA
 * error.
 */
int eik_selftest_local_solve(int device, int64_t count, uint64_t seed, double *max_ulps,
                             double *max_rel);

#ifdef __cplusplus
}
#endif

#endif /* EIK_H */
