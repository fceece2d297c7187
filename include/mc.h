/*
 * mc.h -- C ABI of the B300 per-cell burn library (libmc.so).
 *
 * The operation. A "burn" integrates one zone's reaction network over an
 * operator-split step dt, independently in every cell, with a VODE-style
 * variable-order BDF integrator, caps the number of steps and hands any
 * failure back to the caller as a per-cell status (paper: Software design
 * section, paragraphs 2-4 -- single-zone routines applied over all zones on the
 * GPU, state resident in GPU memory, step cap and failure pass-back, network
 * separate from the integrator, operator-split coupling). The BDF details
 * (variable-coefficient Nordsieck form, modified Newton on I - gamma J,
 * local-error step and order control) are the library's reading of the VODE
 * method the paper cites (Brown, Byrne & Hindmarsh 1989).
 *
 * The network. Species x_i are number fractions (n_i / n, n = total density
 * in cm^-3, held fixed during the burn). Reaction r turns up to two
 * reactant species into up to two product species; each direction has a rate
 * coefficient k = A T^b exp(-C/T) (cm^3/s for two-body, 1/s for one-body), and
 * the forward direction releases dE_eV[r] electron-volts. With energy_eq set,
 * the state also carries the thermal energy per particle-density unit
 * u = (sum x) k_B T / (gamma - 1) and T is recovered from it by the ideal-gas
 * EOS; without it the burn is isothermal at the cell's T (or T = 1 when T is
 * NULL).
 *
 * Memory. Every cell array is structure-of-arrays: x[i * ld + c] is species i
 * of cell c, rate_scale[r * ld + c] the factor of reaction r, stats[k * ld + c]
 * counter k. Arrays are device pointers unless stated otherwise; mc_burn_batch
 * also accepts host pointers (it then stages through library memory and
 * returns after the results are back on the host). The caller owns every cell
 * array; the library owns network constants, scratch and the serving pool.
 *
 * Errors. Calls return an mc_status: MC_OK, or a negative code for bad
 * arguments, allocation or CUDA failures (the message is in mc_last_error(),
 * per thread). A cell whose integration fails is not an error: its status[c]
 * says why and the call still returns MC_OK.
 *
 * Threads and streams. Batch calls are asynchronous on the caller's stream
 * (cudaStream_t passed as void*; NULL = legacy default stream). Network
 * handles are immutable after creation and may be shared by threads. Server
 * calls are thread-safe.
 */
#ifndef MC_H
#define MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mc_status;
#define MC_OK 0
#define MC_PENDING 1
#define MC_E_INVALID (-1)     /* bad argument */
#define MC_E_NOMEM (-2)       /* device or host allocation failed */
#define MC_E_CUDA (-3)        /* a CUDA call failed */
#define MC_E_BUSY (-4)        /* resource in use (e.g. a server still draining) */
#define MC_E_TIMEOUT (-5)     /* a bounded wait ran out */
#define MC_E_NOTFOUND (-6)    /* unknown request id */
#define MC_E_BUDGET (-7)      /* a request can never fit the memory budget */
#define MC_E_UNSUPPORTED (-8) /* network shape outside the compiled range */

/* per-cell status (status[c]) */
#define MC_CELL_OK 0
#define MC_CELL_MAX_STEPS 1   /* step cap reached (the state is at the last accepted time) */
#define MC_CELL_H_UNDERFLOW 2 /* step size fell below the resolution of t */
#define MC_CELL_CONV_FAIL 3   /* 10 consecutive Newton failures */
#define MC_CELL_BAD_INPUT 4   /* non-finite input, T <= 0, n <= 0, or f(y0) not finite */
#define MC_CELL_NONFINITE 5   /* the state stopped being finite */

/* per-cell counters (stats[k * ld + c]) */
#define MC_STAT_STEPS 0       /* accepted steps */
#define MC_STAT_ERR_FAILS 1   /* local-error test failures */
#define MC_STAT_CONV_FAILS 2  /* Newton failures that cut the step */
#define MC_STAT_RHS 3         /* right-hand side evaluations */
#define MC_STAT_JAC 4         /* Jacobian evaluations */
#define MC_STAT_LU 5          /* iteration-matrix factorisations */
#define MC_STAT_NEWTON 6      /* Newton corrections (linear solves) */
#define MC_STAT_ORDER 7       /* BDF order at the end */
#define MC_NSTAT 8

/* integrator variants (mc_burn_opts.variant) */
#define MC_VARIANT_AUTO 0       /* autotuner's choice */
#define MC_VARIANT_PLAIN 1      /* one thread per cell, one launch over the cells */
#define MC_VARIANT_PERSISTENT 2 /* persistent workers pulling cells from a queue */
#define MC_VARIANT_WARP 3       /* persistent, one warp per cell (large networks) */

typedef struct mc_network mc_network;
typedef struct mc_server mc_server;
typedef struct mc_graph mc_graph;

/* Network description, read by mc_network_create (which copies it).
 * react/prod: [n_reactions][2] species indices, -1 for an empty slot (slot 0
 * must be used). A_f..C_r, dE_eV: [n_reactions]. A = 0 disables a direction.
 * n_species + (energy_eq ? 1 : 0) must be <= 40 and n_reactions <= 512. */
typedef struct {
    int32_t n_species;
    int32_t n_elements;   /* informational */
    int32_t n_reactions;
    int32_t energy_eq;    /* 1: carry the energy equation (ideal gas) */
    const int32_t *react;
    const int32_t *prod;
    const double *A_f, *b_f, *C_f;
    const double *A_r, *b_r, *C_r;
    const double *dE_eV;
    double gamma;         /* ratio of specific heats (energy_eq only) */
} mc_network_desc;

/* Integration options. Use mc_burn_opts_default() and override fields. */
typedef struct {
    double rtol;            /* relative tolerance (default 1e-6) */
    double atol;            /* absolute tolerance (default 1e-10) */
    int32_t max_order;      /* highest BDF order, 1..5 (default 5) */
    int32_t max_steps;      /* step cap per cell, counting rejected attempts (default 100000) */
    int32_t lu_precision;   /* 64: FP64 iteration matrix; 32: FP32 matrix and LU, solves
                               refined with FP64 residuals, FP64 history/norm/EOS; a cell
                               whose refinement cannot reach the FP64 solve is retried in
                               FP64 (thread-per-cell) or switches to FP64 factors in place
                               (networks above 16 ODEs, warp-per-cell) */
    int32_t variant;        /* MC_VARIANT_* */
    int32_t block_threads;  /* threads per block, 0 = autotuned */
    int32_t blocks_per_sm;  /* persistent grid = blocks_per_sm x SMs, 0 = autotuned */
    int32_t straggler_steps;/* persistent variant: a cell still running after this many
                               attempts is finished by a whole warp (0 = default 8192,
                               -1 = never) */
    int32_t jacobian;       /* MC_JAC_ANALYTIC (default) or MC_JAC_FD: forward differences,
                               column j = (f(y + d_j e_j) - f(y)) / d_j,
                               d_j = 2^-26 (|y_j| + atol / rtol) (an approximate
                               Jacobian for the paper's per-zone retry, Software design ¶3) */
    int32_t staging;        /* where a thread-per-cell lane's Jacobian and LU are computed:
                               MC_STAGING_SHARED, the whole warp in the warp's shared-memory
                               workspace; MC_STAGING_LANE, the lane alone in its own state;
                               MC_STAGING_AUTO (0) = autotuned, else shared */
} mc_burn_opts;

#define MC_JAC_ANALYTIC 0
#define MC_JAC_FD 1
#define MC_STAGING_AUTO 0
#define MC_STAGING_SHARED 1
#define MC_STAGING_LANE 2

void mc_burn_opts_default(mc_burn_opts *opts);

/* Upload a network: the network is its own object, separate from the
 * integrator that uses it (paper: Software design section, paragraph 4). The
 * description is copied into device constants on the current device; the
 * handle stays valid until mc_network_destroy. Errors: MC_E_INVALID (bad
 * indices or sizes), MC_E_UNSUPPORTED (too many ODEs or reactions),
 * MC_E_NOMEM, MC_E_CUDA. */
mc_status mc_network_create(const mc_network_desc *desc, mc_network **out);
/* Free a network's device constants (paragraph 4). NULL is accepted. The
 * network must not be in use by work still queued on any stream. */
mc_status mc_network_destroy(mc_network *net);
/* ODE count of a network: species plus one for the energy equation (paragraph 4). */
int32_t mc_network_n_ode(const mc_network *net);

/* Burn n_cells cells over dt (seconds) in place: the operator-split reaction
 * step of each zone, one zone per cell, integrated on the GPU and its failure
 * handed back per cell (paper: Software design section, paragraphs 3-4).
 *   x          [n_species][ld] in/out number fractions
 *   T          [ld] in/out temperature (K); required when energy_eq, else the
 *              isothermal temperature of each cell or NULL (T = 1)
 *   ndens      [ld] total density (cm^-3) or NULL (n = 1)
 *   rate_scale [n_reactions][ld] per-cell factor on both directions, or NULL
 *   status     [ld] out per-cell MC_CELL_* code
 *   stats      [MC_NSTAT][ld] out counters, or NULL
 *   stream     cudaStream_t or NULL
 * ld >= n_cells. Device pointers: asynchronous, returns after the launch.
 * Host pointers (all cell arrays on the host): synchronous round trip through
 * library device memory. Errors: MC_E_INVALID, MC_E_NOMEM, MC_E_CUDA.
 * Queue-fed variants (persistent, warp) hand the cells out in decreasing order
 * of a cost key (dt times the error-weighted norm of f at the start): a cell's
 * result does not depend on that order. With 128-thread blocks the persistent
 * variant runs as one cooperative launch in which warps whose queue is drained
 * finish the handed-off cells while the rest of the bulk still runs. */
mc_status mc_burn_batch(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                        double dt, double *x, int64_t ld, double *T, const double *ndens,
                        const double *rate_scale, int32_t *status, int32_t *stats,
                        void *stream);

/* One rung of a retry ladder: the options of one attempt. */
typedef struct {
    mc_burn_opts opts;    /* tolerances, step cap, order, matrix precision, Jacobian */
    int32_t method;       /* MC_METHOD_BDF (the VODE-style integrator) or MC_METHOD_RKC */
} mc_rung;

#define MC_METHOD_BDF 0
#define MC_METHOD_RKC 1   /* explicit Runge-Kutta-Chebyshev, order 2 (Sommeijer, Shampine &
                             Verwer 1998): the integrator the paper offers beside VODE
                             (Software design section, paragraphs 2 and 4); a ladder of one
                             RKC rung is a plain RKC burn */

/* Burn with a retry ladder (paper: Software design section, paragraph 3 --
 * a zone whose integration fails is integrated again under other tolerances
 * or with an approximate Jacobian before the failure is passed back). Every cell is
 * burned with rung 0; a cell whose status is MC_CELL_MAX_STEPS,
 * MC_CELL_H_UNDERFLOW, MC_CELL_CONV_FAIL or MC_CELL_NONFINITE is burned again
 * from its inputs with the next rung, up to n_rungs (1..8). Outputs, status
 * and stats come from the cell's last attempt; rung[c] (int32, may be NULL)
 * receives the rung that produced them. Cell arrays as in mc_burn_batch, device
 * memory only; the failed cells of each rung are compacted into a list that
 * the next rung's launch reads on the device (no host synchronisation).
 * Asynchronous on stream. Errors: MC_E_INVALID, MC_E_NOMEM, MC_E_CUDA. */
mc_status mc_burn_ladder(const mc_network *net, const mc_rung *rungs, int32_t n_rungs, int64_t n_cells, double dt,
                         double *x, int64_t ld, double *T, const double *ndens, const double *rate_scale,
                         int32_t *status, int32_t *stats, int32_t *rung, void *stream);

/* Burn with a constant source term added to every cell's right-hand side:
 * dy/dt = f(y) + s, s = source[i * ld + c] for ODE component i (the species
 * rates, then the energy rate du/dt in eV per unit density and second, with
 * u = (sum x) k_B T / (gamma - 1)). This is the burn inside a step coupled by
 * spectral deferred corrections, where the advective change of each cell is
 * held fixed over the burn (paper: Software design section, paragraph 4, the
 * second coupling mode beside operator splitting). Arguments, layout and
 * errors otherwise as mc_burn_batch (host or device arrays, all alike);
 * source is required. */
mc_status mc_burn_batch_sdc(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells, double dt,
                            double *x, int64_t ld, double *T, const double *ndens, const double *rate_scale,
                            const double *source, int32_t *status, int32_t *stats, void *stream);

/* Rate coefficients k = A T^b exp(-C/T) of the network (paragraph 4's
 * network half; BASELINE workloads' rate form) of every reaction at n
 * temperatures T[c] (device
 * arrays): kf[r * ld + c], kr[r * ld + c] (kr = 0 for irreversible reactions),
 * computed by the burn's own device code (including its table-driven
 * exponential). Asynchronous. Errors: MC_E_INVALID, MC_E_CUDA. */
mc_status mc_network_rates(const mc_network *net, int64_t n, const double *T, double *kf, double *kr,
                           int64_t ld, void *stream);

/* Right-hand side f(y) (and, if jac != NULL, the analytic Jacobian, as the
 * burn's persistent workers evaluate it, one warp per state) -- the network
 * interface the integrator calls (paragraph 4) -- of the
 * burn's ODE system at n states (device arrays): y[i * ld + c] with the
 * energy form's last component u = (sum x) k_B T / (gamma - 1); T is the
 * isothermal temperature (ignored by energy networks, NULL = 1), ndens and
 * rate_scale as in mc_burn_batch; f[i * ld + c], jac[(i * n_ode + j) * ld + c];
 * ok[c] = 0 where the state cannot be evaluated (T <= 0 or non-finite).
 * Asynchronous. Errors: MC_E_INVALID, MC_E_CUDA. */
mc_status mc_network_rhs(const mc_network *net, int64_t n, const double *y, int64_t ld, const double *T,
                         const double *ndens, const double *rate_scale, double *f, double *jac, int32_t *ok,
                         void *stream);

/* Burn without allocating any memory (no counterpart in the paper; a library
 * service). For callers that cannot let a library call cudaMalloc -- programs
 * that give all device memory to their own arena up front and must not see
 * allocations appear later, or latency-critical loops that cannot afford
 * cudaMalloc's implicit synchronisation. Same arguments and results as
 * mc_burn_batch with the persistent variant, except:
 *   - cell arrays must be device memory, and n_cells <= MC_NOALLOC_MAX_CELLS
 *     (larger batches are rejected with MC_E_INVALID before any work);
 *   - its scratch is a fixed file-scope device array of 256 bytes plus 4 bytes
 *     per cell of that maximum (about 4 MB); no straggler hand-off is done;
 *   - the array belongs to the library's device code, which CUDA loads on a
 *     device lazily: the first call on each device (made with that device
 *     current) loads it and looks up the array's device address, and that
 *     first burn may also make the driver reserve local memory for the burn
 *     kernels' per-thread stacks. So make one warm-up call per device before
 *     an arena takes the rest of device memory, and before any stream
 *     capture; the array and the reservation then stay until the process
 *     exits, and later calls allocate nothing (mc_alloc_count does not move);
 *   - every call shares the one array: it clears what must start at zero on
 *     the stream, but calls whose work overlaps on the GPU (different streams,
 *     or another thread) race and corrupt each other's results. */
#define MC_NOALLOC_MAX_CELLS (1 << 20)
mc_status mc_burn_batch_noalloc(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells, double dt,
                                double *x, int64_t ld, double *T, const double *ndens,
                                const double *rate_scale, int32_t *status, int32_t *stats, void *stream);

/* One segment of a mixed batch: cells that share a network, laid out as in
 * mc_burn_batch (device pointers), and their own burn interval dt (seconds;
 * 0 takes the dt passed to the call), so networks with different time scales
 * share one launch. */
typedef struct {
    const mc_network *net;
    int64_t n_cells;
    int64_t ld;
    double *x;
    double *T;
    const double *ndens;
    const double *rate_scale;
    int32_t *status;
    int32_t *stats;
    double dt;
} mc_segment;

/* Burn several segments (different networks, uneven stiffness, each with its
 * own dt) in ONE
 * persistent launch: workers pull cells from per-network queues, and a lane
 * whose cell finishes takes the next cell (paper: divergence between zones,
 * Software design section, paragraph 3). Asynchronous on stream. */
mc_status mc_burn_mixed(const mc_segment *segs, int32_t n_segs, const mc_burn_opts *opts,
                        double dt, void *stream);

/* Capture mc_burn_mixed for fixed segments into a CUDA graph (paragraph 3's
 * zone loop as one replayable unit of GPU work: queue reset,
 * persistent launch, counter reduction) and replay it with mc_graph_launch.
 * The segment arrays must stay allocated while the graph exists; their
 * contents may change between launches. totals (may be NULL) receives, after
 * each replay, the MC_NSTAT counters summed over all cells (device int64[8]). */
mc_status mc_graph_create(const mc_segment *segs, int32_t n_segs, const mc_burn_opts *opts,
                          double dt, int64_t *totals, void *stream, mc_graph **out);
/* Replay a captured mixed burn on stream (asynchronous). Errors: MC_E_INVALID, MC_E_CUDA. */
mc_status mc_graph_launch(mc_graph *g, void *stream);
/* Free a graph and the scratch its replays use (waits for the device). */
mc_status mc_graph_destroy(mc_graph *g);

/* Autotune the zone loop of paragraph 3 on this GPU: measure every launch
 * shape (plain or persistent x threads per block x
 * persistent blocks per SM) on a sample of n_sample cells (device arrays laid
 * out as in mc_burn_batch; they are copied, not modified) and keep the fastest
 * for this network size and opts->lu_precision: later burns whose shape
 * fields are 0 use it. The winner is written to *best (may be NULL) and
 * appended to the JSON-lines file named by the MC_AUTOTUNE_CACHE environment
 * variable, which is read back on first use. Synchronous. */
mc_status mc_autotune(const mc_network *net, const mc_burn_opts *opts, int64_t n_sample, double dt,
                      const double *x, int64_t ld, const double *T, const double *ndens, void *stream,
                      mc_burn_opts *best);

/* ---------------------------------------------------------------- serving */
/* A server (paper: state resident in GPU memory, Software design section,
 * paragraph 3) admits burn requests in arrival order while the device bytes
 * they need stay within hbm_budget_bytes: each request's state in pooled
 * device memory ((n_species + 2) doubles and one int per cell, see
 * mc_request_bytes) plus the growth of the library scratch of the stream it
 * runs on (the server keeps 8 streams; scratch is per stream and never
 * shrinks, so each stream's high-water mark stays charged). An admitted
 * request's state is copied into the pool, burned with its own options on
 * its stream, its failed cells counted on the device, and the results copied
 * back to the caller's buffers. Requests that arrive while others are on the
 * GPU start as soon as memory and a stream are free, so their work overlaps on
 * the device (continuous batching); a host thread does admission and
 * completion, the GPU work is enqueued outside the server's lock, and no device
 * code waits on the host. Server calls are thread-safe. */
typedef struct {
    int32_t state;          /* MC_PENDING or MC_OK */
    int32_t n_failed;       /* cells with status != MC_CELL_OK */
    int64_t n_cells;
    double t_submit;        /* seconds on the server's monotonic clock */
    double t_admit;
    double t_done;
    double gpu_start;       /* seconds from the server's creation on the GPU's clock: */
    double gpu_end;         /* when the request's work started and ended on its stream */
} mc_request_info;

/* opts: the server's default options for requests that pass none. */
mc_status mc_server_create(int32_t device, uint64_t hbm_budget_bytes, const mc_burn_opts *opts,
                           mc_server **out);
/* Bytes a request of n_cells charges against the budget: its pooled state and
 * the stream scratch its burn needs (either pointer may be NULL). */
mc_status mc_request_bytes(const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                           uint64_t *state_bytes, uint64_t *scratch_bytes);
/* Queue a request (paper: Software design section, paragraph 3, one zone's
 * burn handed to the GPU). opts may be NULL (the server's). Cell arrays as in
 * mc_burn_batch (host or device memory; rate_scale is not supported here).
 * The caller must not touch them until mc_request_poll reports MC_OK. Never
 * blocks on the GPU. Errors: MC_E_BUDGET if the request alone exceeds the
 * budget, MC_E_INVALID, MC_E_BUSY while the server shuts down. */
mc_status mc_request_submit(mc_server *srv, const mc_network *net, const mc_burn_opts *opts, int64_t n_cells,
                            double dt, double *x, int64_t ld, double *T, const double *ndens,
                            int32_t *status, uint64_t *req_id);
/* MC_PENDING while in flight, MC_OK once results are in the caller's buffers
 * (info filled in either case when non-NULL); the request's own error code and
 * message if its work failed; MC_E_NOTFOUND for an unknown id. */
mc_status mc_request_poll(mc_server *srv, uint64_t req_id, mc_request_info *info);
/* Wait (bounded by timeout_s) until every submitted request is done. */
mc_status mc_server_drain(mc_server *srv, double timeout_s);
/* Drain (bounded, 600 s) and free. MC_E_TIMEOUT if work was still running. */
mc_status mc_server_destroy(mc_server *srv);

/* ---------------------------------------------------------------- misc */
/* Library services with no counterpart in the paper. */
/* Message of this thread's last error (empty when none); owned by the library. */
const char *mc_last_error(void);
/* ABI version of this header and library. */
int32_t mc_version(void);
/* Kernel launches issued by this thread since the last reset (for accounting). */
int64_t mc_launch_count(int32_t reset);
/* Device and pinned-host allocations the library has made in this process,
 * all threads (network uploads, scratch growth, host-array staging, serving
 * pool, autotuner copies). mc_burn_batch_noalloc never adds to it. */
int64_t mc_alloc_count(void);
/* Measure the fused multiply-add rate (TFLOP/s, 2 flops per FMA) of the
 * current device in FP64 and FP32 with dependent-free FMA chains over every SM
 * (about 10 ms each): the ceiling this ALU-bound burn is reported against.
 * Either pointer may be NULL. Synchronous. Errors: MC_E_CUDA, MC_E_NOMEM. */
mc_status mc_probe_fma_rate(double *tflops_fp64, double *tflops_fp32);

/* Bounds-check build. libmc_check.so is this library compiled with
 * -DMC_BOUNDS_CHECK: every cell index, list position and straggler-record
 * index a burn kernel computes is tested before the access it guards; a
 * refused access is counted (the first one recorded) and skipped instead of
 * faulting, and mc_burn_batch, mc_burn_batch_sdc and mc_burn_ladder count each
 * cell's final store and verify on the device, after the call, that every
 * cell was stored exactly once (the queue handed every cell out once; the
 * hand-off, retry lists and rungs lost and duplicated none). Store counting
 * assumes one such call at a time per device. In the normal build nothing is
 * checked and the report has enabled = 0. */
typedef struct mc_bounds_info {
  int32_t enabled;          /* 1 in the bounds-check build */
  uint32_t refused;         /* accesses refused since the last reset */
  int32_t first_site;       /* site of the first refused access (0: none): 1 cell load, 2 cell
                               store, 3 list read, 4 list push, 5 record, 6 warp-form load, 7 RKC */
  int32_t pad;
  int64_t first_index;      /* its index */
  int64_t first_bound;      /* and bound */
  int64_t calls_checked;    /* calls whose stores were verified */
  int64_t cells_checked;    /* cells over those calls */
  int64_t cells_not_once;   /* cells of those calls not stored exactly once */
} mc_bounds_info;
/* The device's record (synchronises the device). Errors: MC_E_INVALID (null
 * out), MC_E_CUDA. */
mc_status mc_bounds_report(int32_t device, mc_bounds_info *out);
/* Zero the device's record (synchronises the device). */
mc_status mc_bounds_reset(int32_t device);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
