/*
 * zbus.h -- C ABI of libzbus, a batched three-phase Z-bus power-flow solver
 * for one NVIDIA GB300 (sm_103a).
 *
 * The method is the current-injection fixed point of arxiv 2605.14103,
 * Sec. II-B:
 *
 *     v_b^{k+1} = Z i(v_b^k, S_b^wye, S_b^del) + w
 *
 * where Z is the reduced bus impedance of the non-slack phases, w the no-load
 * voltage (the paper's v_0) and i(.) the current injection of constant-power
 * wye and delta loads.  Many load scenarios b share one Z.
 *
 * Conventions shared by every call:
 *   - Complex numbers are interleaved (re, im) doubles.
 *   - Unknowns: the non-slack bus-phases of the admittance matrix, in
 *     ascending global index order; n of them.  For a feeder whose bus k
 *     occupies global indices 3k, 3k+1, 3k+2 with bus 0 the slack, unknown
 *     j = 3(k-1) + phase.
 *   - Loads are consumption (pu).  A wye slot j draws conj(S_wye_j / v_j).
 *     A delta load of a bus sits in the bus's three slots in branch order
 *     (ab, bc, ca); branch xy draws conj(S_xy / (v_x - v_y)) out of phase x
 *     and returns it into phase y.  Delta loads require n to be a multiple
 *     of 3 (three consecutive unknowns per bus).  A slot with S = 0 draws
 *     nothing.
 *   - Scenario arrays are scenario-major: element (b, j) of a [B][n] complex
 *     array is at offset 2*(b*n + j) doubles.
 *   - Device pointers are plain CUDA device addresses (for example a torch
 *     tensor's data_ptr()); streams are cudaStream_t passed as void* (NULL is
 *     the legacy default stream).
 *   - Calls return a zbus_status; on an argument error nothing is launched and
 *     outputs are untouched.  zbus_last_error() gives a message for the last
 *     failing call of the calling thread.
 *   - A network handle is not thread-safe: calls on one handle must not run
 *     concurrently from several host threads.
 */
#ifndef ZBUS_H
#define ZBUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zbus_network_s* zbus_network;

typedef enum {
  ZBUS_OK = 0,
  ZBUS_ERR_ARG = 1,         /* invalid argument; nothing was launched */
  ZBUS_ERR_SINGULAR = 2,    /* Y_LL is singular to working precision */
  ZBUS_ERR_OOM = 3,         /* device allocation failed or budget exceeded */
  ZBUS_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  ZBUS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  ZBUS_ERR_DEVICE = 6,      /* a kernel reported an internal error word */
  ZBUS_ERR_UNSUPPORTED = 7, /* option not available for this network / device */
  ZBUS_ERR_SOURCE = 8       /* zbus_serve: the request source reported a failure */
} zbus_status;

typedef enum {
  ZBUS_FP64 = 0,              /* plain map, FP64 on the CUDA cores */
  ZBUS_MIXED_BF16X2 = 1,      /* defect form, Z as BF16 hi+lo on tensor cores */
  ZBUS_MIXED_FP16_SCALED = 2, /* defect form, Z as row-scaled FP16 hi+lo */
  ZBUS_TREE_SWEEP = 3         /* defect form, Z applied as a backward / forward
                                 sweep over a radial feeder (FP32, O(n) per
                                 scenario instead of O(n^2)); radial networks
                                 only, else ZBUS_ERR_UNSUPPORTED */
} zbus_precision;

typedef enum {
  ZBUS_CONV_MAXABS = 0,  /* max_j |v_j^k - v_j^{k-1}| <= tol */
  ZBUS_CONV_SUMMAG = 1   /* | sum_j |v_j^k| - sum_j |v_j^{k-1}| | <= tol (Sec. II-B) */
} zbus_conv_rule;

typedef struct {
  int32_t precision;       /* zbus_precision */
  int32_t conv_rule;       /* zbus_conv_rule */
  double mismatch_tol;     /* mixed modes: a converged scenario must also have
                              max_j |v_j conj(r_j)| <= mismatch_tol (FP64);
                              <= 0 selects 1e-6 */
  int32_t max_correction;  /* mixed modes: a scenario that met the stop rule
                              but fails the FP64 mismatch test gets up to
                              max_correction FP64 correction sweeps (r =
                              i(v) - Y_LL v - Y_Ls v_s in FP64, v += Z r with
                              the FP64 Z, then the test again); it keeps its
                              flag once the test passes and loses it if none
                              does.  Each sweep counts as an iteration.
                              <= 0: none (the flag is cleared at once);
                              default 8 */
  int32_t profile;         /* 1: run the sweeps from the host with CUDA events
                              around every kernel on cuda_stream, for
                              zbus_last_profile; 0: device-resident loop */
  int32_t fp32_start;      /* mixed modes (BF16X2, FP16_SCALED, TREE_SWEEP),
                              cold starts (V_init NULL): 1 (default) = a scenario's
                              first sweeps form the defect residual in FP32
                              (block products with the FP32 part of Y, load
                              currents at the FP32 voltage) as long as its max
                              |r| exceeds 2^-20 of its largest line or load
                              current, falls from sweep to sweep and its step
                              exceeds tol, then double-float to the stop; no
                              scenario stops on an FP32 sweep, so the fixed
                              point and the stop rule are those of the
                              double-float residual.  0 = double-float from
                              the first sweep.  Per scenario: a result does
                              not depend on the batch around it. */
  int32_t reserved_i;
  double reserved[3];
} zbus_solve_opts;

/* Fill *opts with the defaults (FP64, max-step rule). */
void zbus_solve_opts_default(zbus_solve_opts* opts);

/*
 * zbus_network_create -- set up one network on the current CUDA device.
 *
 * Sec. II-B: separates slack and non-slack phases and precomputes the reduced
 * bus impedance.  On the device, in FP64: dense Y_LL and Y_Ls from the COO
 * entries (duplicates summed), Z = Y_LL^{-1} by Gauss-Jordan elimination with
 * partial pivoting, w = -Z Y_Ls v_s, and the operand layouts of every
 * precision.
 *
 *   n_total       number of bus-phases including the three slack phases (>= 4)
 *   nnz           number of COO entries (>= 1)
 *   row, col      host int32[nnz], 0 <= row, col < n_total
 *   val_reim      host double[2*nnz], complex admittance entries (pu)
 *   slack_idx     host int32[3], distinct global indices of the slack phases
 *   v_slack_reim  host double[6], complex slack phase voltages (pu)
 *   cuda_stream   stream for the setup work; the call returns after it finished
 *   out           receives the handle (owned by the library until destroy)
 *
 * Returns ZBUS_ERR_SINGULAR if a pivot is zero or not finite, ZBUS_ERR_OOM if
 * device memory runs out.
 */
zbus_status zbus_network_create(int32_t n_total, int64_t nnz,
                                const int32_t* row, const int32_t* col,
                                const double* val_reim,
                                const int32_t* slack_idx,
                                const double* v_slack_reim,
                                void* cuda_stream, zbus_network* out);

/*
 * zbus_network_create_phased -- zbus_network_create for a feeder whose buses
 * carry any subset of the phases (single- and two-phase laterals).
 *
 *   bus_phase  host int32[n_total]: 3 * bus + phase (phase 0, 1, 2 = a, b, c)
 *              of every global index; the slack is bus 0 and bus_phase of
 *              slack_idx[p] must be p; every value at most once.
 *
 * The other arguments are those of zbus_network_create.  The device solves
 * the network padded to three phase slots per bus, an absent phase an
 * isolated node with a unit self-admittance (its voltage stays 0): the fixed
 * point of Sec. II-B on the present phases.  Every array of zbus_solve and
 * zbus_power_mismatch is then [B][n] over the present non-slack phases in
 * ascending global index (n = zbus_network_size); zbus_network_get_z gives Z
 * and w on those unknowns.  A delta entry sits at the branch's first phase
 * (ab, bc, ca) and is a load only where the branch's second phase is present
 * (other entries are ignored).  zbus_solve_batched, zbus_serve,
 * zbus_autotune and zbus_solve_noalloc return ZBUS_ERR_UNSUPPORTED for such
 * a network.  Returns ZBUS_ERR_ARG for a map that breaks these rules.
 */
zbus_status zbus_network_create_phased(int32_t n_total, int64_t nnz,
                                       const int32_t* row, const int32_t* col,
                                       const double* val_reim, const int32_t* slack_idx,
                                       const double* v_slack_reim, const int32_t* bus_phase,
                                       void* cuda_stream, zbus_network* out);

/* Release a network and every device buffer it owns.  NULL is ignored.  The
 * caller must make sure no work of this handle is still running. */
void zbus_network_destroy(zbus_network net);

/* Number of unknowns n (non-slack bus-phases) of a network; -1 for NULL. */
int32_t zbus_network_size(zbus_network net);

/*
 * zbus_network_get_z -- copy the device-formed Z (row-major [n][n] complex)
 * and w ([n] complex) into caller device buffers, on cuda_stream.  Either
 * output may be NULL.
 */
zbus_status zbus_network_get_z(zbus_network net, double* Z_out, double* w_out,
                               void* cuda_stream);

/*
 * zbus_network_reserve -- grow the handle's scratch space for batches of up to
 * B scenarios in the given precision, so that later zbus_solve calls of that
 * size allocate nothing.  Synchronous.
 */
zbus_status zbus_network_reserve(zbus_network net, int64_t B, int32_t precision);

/*
 * zbus_solve -- batched fixed point over B scenarios (Sec. II-B).
 *
 *   S_wye, S_delta  device, [B][n] complex, consumption (pu); either may be
 *                   NULL for "no loads of that kind"
 *   V_init          device [B][n] complex warm start, or NULL for v^0 = w
 *   tol             stop tolerance of the chosen rule (pu), >= 0
 *   max_iter        iteration cap, >= 1
 *   opts            NULL for the defaults
 *   V_out           device [B][n] complex, the last iterate of every scenario
 *   iters           device int32[B], maps performed (including the one that
 *                   met tol)
 *   converged       device uint8[B], 1 if the rule was met (and, in the mixed
 *                   modes, the FP64 mismatch test passed)
 *   cuda_stream     all work is enqueued on this stream; results are valid
 *                   after it synchronises.  Scratch grows on demand (a
 *                   synchronous allocation) unless reserved beforehand.
 *
 * The array arguments are all device memory or all host memory (pinned or
 * pageable; a mix returns ZBUS_ERR_ARG).  With host memory the batch is
 * solved in chunks staged through the device: the host-to-device copy of one
 * chunk and the device-to-host copy of the previous one run on copy streams
 * while the sweeps of another chunk run on cuda_stream (pinned memory lets
 * them overlap), and cuda_stream waits for the last copy.  Results are the
 * same bit for bit as with device buffers.
 *
 * Non-convergence is reported by the flags, not by the status.  V_out may
 * alias V_init.  B = 0 is a no-op.
 *
 * ZBUS_TREE_SWEEP (the sparse application of Z the paper leaves to future
 * work, Sec. II-B): for a feeder whose buses form a tree hanging off the slack
 * with reciprocal branches, Y_LL^{-1} r is a backward sweep (subtree sums of
 * r) followed by a forward sweep (path sums of branch impedances times those
 * sums); the defect residual stays exact (shunts included), so the fixed
 * point is that of the other forms.  Returns ZBUS_ERR_UNSUPPORTED for a meshed
 * or non-reciprocal network, or one above 3592 buses.
 */
zbus_status zbus_solve(zbus_network net, int64_t B,
                       const double* S_wye, const double* S_delta,
                       const double* V_init, double tol, int32_t max_iter,
                       const zbus_solve_opts* opts,
                       double* V_out, int32_t* iters, uint8_t* converged,
                       void* cuda_stream);

/* One feeder of a batched solve: its network, scenario count and buffers
 * (same meaning and layout as the arguments of zbus_solve). */
typedef struct {
  zbus_network net;
  int64_t B;
  const double* S_wye;
  const double* S_delta;
  const double* V_init;
  double* V_out;
  int32_t* iters;
  uint8_t* converged;
} zbus_batch_item;

/*
 * zbus_solve_batched -- several feeders of uneven size and scenario count in
 * one solve (Sec. II-B fixed point for each).  In the mixed precisions the
 * sweeps of all feeders run as one set of kernels per sweep (one persistent
 * tensor-core contraction over the tiles of every feeder) inside one CUDA
 * graph WHILE loop; each feeder's scenarios stop independently.  In FP64 the
 * feeders are solved one after another.  A network may appear at most once
 * per call.  Results equal those of zbus_solve on each feeder alone.
 */
zbus_status zbus_solve_batched(const zbus_batch_item* items, int32_t n_items, double tol,
                               int32_t max_iter, const zbus_solve_opts* opts,
                               void* cuda_stream);

/*
 * zbus_autotune -- time every compiled tensor-core contraction variant (N-tile
 * and pipeline depth) of opts->precision on this workload (reps timed solves
 * each, after one warm-up) and record the fastest for its size bucket (next
 * powers of two of the largest feeder's n and of the total scenario count).
 * The table persists in $ZBUS_TUNE_CACHE, else zbus_tune.json beside the
 * library, and is consulted by every later mixed-precision solve.  The
 * winner is returned in *best_BN / *best_stages (either may be NULL).
 * Project-written; the paper has no counterpart.
 */
zbus_status zbus_autotune(const zbus_batch_item* items, int32_t n_items,
                          const zbus_solve_opts* opts, double tol, int32_t max_iter,
                          int32_t reps, void* cuda_stream, int32_t* best_BN,
                          int32_t* best_stages);

/*
 * zbus_tune_variants -- the compiled tensor-core contraction variants of a
 * mixed precision (ZBUS_MIXED_BF16X2 or ZBUS_MIXED_FP16_SCALED): up to `max`
 * (N-tile, pipeline stages) pairs into the caller's host arrays BN[] and
 * stages[] (either may be NULL to count only).  Returns the number of
 * variants, 0 for a precision without tensor-core tiles, -1 for max < 0.
 */
int32_t zbus_tune_variants(int32_t precision, int32_t* BN, int32_t* stages, int32_t max);

/*
 * zbus_tune_set -- record the contraction variant (BN, stages) for the size
 * bucket of (max_n, total_B), the same buckets as zbus_autotune, in this
 * process's table (not written to the cache file).  Every later
 * mixed-precision solve or serving loop in that bucket uses it.  BN = 0
 * removes the entry (the built-in choice applies again).  ZBUS_ERR_ARG for
 * a precision without tensor-core tiles, max_n or total_B below 1, or a
 * (BN, stages) pair that is not compiled (zbus_tune_variants).
 * Project-written; the paper has no counterpart.
 */
zbus_status zbus_tune_set(int32_t precision, int32_t max_n, int64_t total_B, int32_t BN,
                          int32_t stages);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over a pool of networks with continuous batching.
 * ------------------------------------------------------------------------- */

/* One request: B scenarios of one pool feeder. */
typedef struct {
  int32_t feeder;          /* index into the pool */
  int64_t B;               /* scenarios, 1 .. the feeder's slot capacity */
  const double* S_wye;     /* device [B][n] complex or NULL; valid until completion */
  const double* S_delta;   /* device [B][n] complex or NULL */
  double* V_out;           /* device [B][n] complex, or NULL: results stay in a
                              library buffer passed to the sink (valid during
                              the sink call only) */
  int32_t* iters;          /* device [B] or NULL (with V_out NULL) */
  uint8_t* converged;      /* device [B] or NULL (with V_out NULL) */
  int32_t warm_start;      /* 1: start from the feeder's last converged voltage
                              (kept on the device), else from w */
  int32_t reserved0;
  uint64_t tag;            /* caller's identifier */
  double t_arrival;        /* arrival time, seconds on the serving clock */
} zbus_request;

/* Outcome of one request, passed to the sink. */
typedef struct {
  zbus_status status;      /* ZBUS_OK, or ZBUS_ERR_ARG for a request that can
                              never fit (B above the slot capacity, bad feeder) */
  int32_t n_converged;     /* scenarios flagged converged (after the FP64 test) */
  int32_t max_iters;       /* largest iteration count of its scenarios */
  int32_t operands_formed; /* 1: its admission formed the feeder's operands
                              (a miss of the serving loop's operand cache) */
  double t_admit;          /* seconds on the serving clock */
  double t_done;           /* results complete on the device */
  const double* V;         /* device [B][n] results (V_out or the library buffer) */
  const int32_t* iters;    /* device [B] */
  const uint8_t* converged;/* device [B] */
} zbus_request_result;

/* Polled by the serving loop with the current serving-clock time (seconds
 * since the loop started): return 1 and fill *req if a request is ready, 0 if
 * none is ready now, -1 when no further request will come, -2 (or below) if
 * the source failed: no further request is taken, the requests it had
 * delivered are still served, and zbus_serve returns ZBUS_ERR_SOURCE. */
typedef int32_t (*zbus_request_source)(void* user, double now, zbus_request* req);
/* Called once per request when its results are complete on the device. */
typedef void (*zbus_completion_sink)(void* user, const zbus_request* req,
                                     const zbus_request_result* res);

typedef struct {
  uint64_t hbm_budget_bytes;   /* device bytes for the pool's operands plus the
                                  slot state of every feeder */
  int32_t max_slots;           /* upper bound of scenario slots per feeder */
  int32_t precision;           /* ZBUS_MIXED_FP16_SCALED, ZBUS_MIXED_BF16X2 or
                                  ZBUS_TREE_SWEEP (every pool network radial) */
  int32_t conv_rule;
  int32_t max_iter;
  double tol;
  double mismatch_tol;         /* <= 0 selects 1e-6 */
  int32_t max_admit_per_sweep; /* <= 0: unlimited */
  int32_t max_correction;      /* FP64 correction sweeps per scenario, as in
                                  zbus_solve_opts (<= 0: none, the flag of a
                                  scenario above mismatch_tol is cleared) */
  int32_t fp32_start;          /* as in zbus_solve_opts, for requests without
                                  a warm start (0: double-float throughout) */
} zbus_serve_config;

/*
 * zbus_serve -- run the request loop until the source signals the end and
 * every admitted request has completed.  Each loop pass admits pending
 * requests into free scenario slots of their feeder (first fit, in arrival
 * order), runs one sweep of the grouped mixed-precision engine over every
 * active slot of every feeder, and completes the requests whose scenarios
 * have all stopped (FP64 mismatch test and correction sweeps, results to the
 * caller, sink call).
 * Requests that arrive while others are on the GPU join at the next sweep
 * (continuous batching); per-scenario arithmetic does not depend on the mix,
 * so a result is the same alone and in the mix.
 *
 * HBM budget (hbm_budget_bytes): every feeder gets the same slot capacity,
 * the largest multiple of 128 (<= max_slots) whose state, over all feeders,
 * leaves room for the largest feeder's operands while they are formed
 * (ZBUS_ERR_OOM if not even 128 do).  The rest of the budget is an operand
 * cache (the Z_LL cache): a resident feeder holds its tensor-core Z and the
 * FP64 3M copies of Z (for the correction sweeps); its complex FP64 Z is
 * released once those are formed.  At the start the pool's feeders are made
 * resident in pool order while they fit; the others release their dense
 * operands.  A request for a feeder that is not resident evicts idle
 * feeders (no request in flight), least recently used first, until the
 * feeder's operands can be formed on the device (Z_LL^-1 again by
 * Gauss-Jordan, then its copies), and waits while they cannot; requests of
 * other feeders are admitted meanwhile.  Released operands of a pool network
 * are formed again on demand by any later call that needs them.  Each feeder
 * keeps its last converged voltage for warm starts.  Runs on the calling
 * thread; the callbacks run on it too.
 */
zbus_status zbus_serve(const zbus_serve_config* cfg, zbus_network* pool, int32_t n_pool,
                       zbus_request_source src, zbus_completion_sink sink, void* user,
                       void* cuda_stream);

/*
 * zbus_serve_footprint -- what zbus_serve counts against its HBM budget for
 * one pool network in a precision: the operand bytes it holds while resident
 * in the operand cache, the extra bytes a formation needs while it runs, and
 * the bytes of one scenario slot.  Any output may be NULL.  Host only.
 * Project-written sizing query.
 */
zbus_status zbus_serve_footprint(zbus_network net, int32_t precision, uint64_t* operand_bytes,
                                 uint64_t* formation_bytes, uint64_t* slot_bytes);

/*
 * zbus_power_mismatch -- per-scenario FP64 power mismatch of given voltages,
 * max_j |v_j conj((Y_LL v + Y_Ls v_s)_j - i_j(v))|, computed with the sparse
 * admittance matrix (never with Z).  V, S_* device [B][n] complex; out device
 * double[B].
 */
zbus_status zbus_power_mismatch(zbus_network net, int64_t B, const double* V,
                                const double* S_wye, const double* S_delta,
                                double* out, void* cuda_stream);

/*
 * zbus_last_profile -- per-sweep kernel times of the last zbus_solve on this
 * handle that ran with opts.profile = 1.  Call after that solve's stream has
 * synchronised.  For sweep k < min(max_n, sweeps): ms[3k + 0..2] receive the
 * durations (milliseconds, CUDA events) of the load-current / residual
 * kernel, the contraction and the convergence kernel; active[k] the number of
 * scenarios the sweep processed.  *sweeps receives the number of sweeps
 * launched (the loop runs max_iter sweeps; those after the last active one
 * have active[k] = 0).  Any output may be NULL.
 */
zbus_status zbus_last_profile(zbus_network net, int32_t max_n, float* ms, int32_t* active,
                              int32_t* sweeps);

/*
 * zbus_solve_noalloc -- the plain FP64 solve (same results as zbus_solve with
 * precision ZBUS_FP64) for callers that cannot allocate device memory while
 * they solve: processes whose device memory is owned by another allocator,
 * real-time loops that forbid allocation after start-up, plug-in hosts that do
 * not let plug-ins allocate.  The paper has no counterpart; this is a
 * property of this library's interface.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (solve context, active list, per-tile partials, contraction operands) lives
 * in one static 16 MiB device array.  zbus_network_create loads that array on
 * its device and looks up its address (with that device current), so every
 * device on which a network was created holds the 16 MiB from then until the
 * process exits, and this call itself loads nothing.  The network must exist
 * already (create it at start-up, before any stream capture).  The sweeps are
 * launched from the host (max_iter sweeps; once no scenario is active the
 * remaining launches return at once).
 *
 *   arguments as zbus_solve, with conv_rule (zbus_conv_rule) in place of
 *   opts, but device memory only: a host array (pinned or pageable) returns
 *   ZBUS_ERR_ARG, launching nothing.  Also ZBUS_ERR_ARG, launching nothing,
 *   when the batch needs more than the 16 MiB: about 16 MiB / (24 n_pad +
 *   16 ceil(n/48) + 5) bytes per scenario, n_pad = n rounded up to a multiple
 *   of 48 (about 1790 scenarios for n = 381).  Partial-phase networks:
 *   ZBUS_ERR_UNSUPPORTED.  After this call zbus_last_device_status reports
 *   ZBUS_OK (the FP64 sweeps have no device-side waits).
 *
 * All calls share the array and it keeps the last call's contents; every call
 * rewrites what it reads, but calls that overlap on the GPU (other streams or
 * other host threads) race on it.
 */
zbus_status zbus_solve_noalloc(zbus_network net, int64_t B,
                               const double* S_wye, const double* S_delta,
                               const double* V_init, double tol, int32_t max_iter,
                               int32_t conv_rule,
                               double* V_out, int32_t* iters, uint8_t* converged,
                               void* cuda_stream);

/*
 * zbus_solve_adjoint -- gradient of a real loss L(v*) with respect to the
 * loads, v* a converged solution of the Sec. II-B fixed point v = Z i(v, S) + w
 * (the paper presents the solver as a component of GPU learning pipelines,
 * Sec. I and the conclusion; this makes the solve differentiable).  The
 * gradient is taken through the fixed-point condition (implicit function
 * theorem), not through the iterations:
 *     lambda = G + A^T mu,   mu = Z^T conj(lambda)   (iterated from mu = 0),
 *     dL/dS = D^T mu,
 * with di = A conj(dv) + D conj(dS) the linearised load current at v* (wye
 * slot j: A_jj = conj(S_j / v_j^2), D_jj = -1 / conj(v_j); delta branch
 * x -> y, u = v_x - v_y: conj(S / u^2) in A on (x,x), (y,y) and its negative on
 * (x,y), (y,x); -1 / conj(u), +1 / conj(u) at rows x, y of D).  FP64 throughout
 * (the 3M contraction of the plain method with Z^T); the sweeps run in a
 * device-side loop like the solve.
 *
 * Complex gradients follow the convention of complex autograd:
 * grad = dL/dRe + j dL/dIm, so dL = Re(sum conj(grad) dS).
 *
 *   S_wye, S_delta  device [B][n] complex loads of the solve (either NULL)
 *   V               device [B][n] complex converged voltages (e.g. V_out of
 *                   zbus_solve)
 *   G               device [B][n] complex dL/dV
 *   tol             stop when max_j |mu^k_j - mu^{k-1}_j| <= tol after G_b
 *                   is scaled to max_j |G_bj| = 1 (a tolerance relative to
 *                   each scenario's loss gradient); >= 0
 *   max_iter        iteration cap, >= 1
 *   opts            NULL, or opts->precision: ZBUS_FP64 (default; the dense
 *                   Z^T sweeps above) or ZBUS_TREE_SWEEP (radial networks
 *                   with reciprocal branches: the defect iteration
 *                   rho = conj(G/s + A^T mu) - Y_LL^T mu, mu += T^T rho, with
 *                   Y_LL^T mu from the sparse branch blocks and T^T the
 *                   backward / forward sweep of the transposed series network,
 *                   O(n) per scenario and sweep, FP64, one CTA per scenario;
 *                   same fixed point; ZBUS_ERR_UNSUPPORTED for a meshed
 *                   network); other fields are ignored
 *   dS_wye          device [B][n] complex dL/dS_wye, or NULL; defined for
 *                   every slot (the sensitivity to adding a load there)
 *   dS_delta        device [B][n] complex dL/dS_delta, or NULL; slot x is the
 *                   branch x -> next phase; zero where the branch lacks its
 *                   second phase (partial-phase networks)
 *   iters           device int32[B] adjoint sweeps performed
 *   converged       device uint8[B] 1 where the stop rule was met; a
 *                   scenario whose V is not a stable fixed point does not
 *                   converge and its gradient is not to be used
 *   cuda_stream     all work is enqueued on this stream
 *
 * Device buffers only (ZBUS_ERR_ARG otherwise).  The first call on a network
 * forms Z^T (three n_pad x n_pad FP64 arrays kept with the handle); scratch
 * grows on demand (synchronous).  Shares the handle's solve scratch, so it
 * must not overlap a solve of the same handle on another stream.  Works on
 * partial-phase networks.  B = 0 is a no-op.
 */
zbus_status zbus_solve_adjoint(zbus_network net, int64_t B,
                               const double* S_wye, const double* S_delta,
                               const double* V, const double* G,
                               double tol, int32_t max_iter,
                               const zbus_solve_opts* opts,
                               double* dS_wye, double* dS_delta,
                               int32_t* iters, uint8_t* converged,
                               void* cuda_stream);

/*
 * zbus_last_device_status -- the errors the device detected during the last
 * solve on net (the error word its kernels set instead of hanging or
 * faulting).  Synchronises cuda_stream first, so the solve must have been
 * enqueued on it.  ZBUS_OK if the solve ran clean (or was FP64, which has no
 * device-side waits); ZBUS_ERR_TIMEOUT if a bounded wait of the tensor-core
 * pipeline gave up (its results are then not to be used); ZBUS_ERR_DEVICE
 * for any other error word.  The next solve clears the word.  Project-
 * written; the paper has no counterpart.
 */
zbus_status zbus_last_device_status(zbus_network net, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Transmission grids: batched Newton-Raphson power flow (Sec. II-A).
 *
 * State x_b = [theta_Theta; |V|_Q] (angles of the PV and PQ buses,
 * magnitudes of the PQ buses), mismatch F_b = [P_calc - P on Theta;
 * Q_calc - Q on Q], S_calc = V o conj(Y V) (eqs. 1-2); Newton steps
 * J dx = -F (eq. 3) solved by restarted GMRES with Jacobian-vector products
 * and the block lower-triangular fast-decoupled preconditioner of eqs. 7-9
 * (B' = -Im(Y)[Theta,Theta], B'' = -Im(Y)[Q,Q] with eps I added,
 * G_Q,Theta = -Re(Y)[Q,Theta]), FP64.  B' + eps I and B'' + eps I are
 * applied through sparse LU factors formed at network creation.
 * ------------------------------------------------------------------------ */
typedef struct zbus_nr_network_s* zbus_nr_network;

/* Arithmetic of the Newton direction.  ZBUS_NR_FP64: everything in FP64
 * (the paper's solver).  ZBUS_NR_MIXED: GMRES, the Jacobian-vector products
 * and the preconditioner in FP32 (dot products summed in FP64), while the
 * mismatch, the state update and the stop test stay FP64: the direction is
 * an inexact Newton step, the converged solution that of F = 0 in FP64. */
typedef enum { ZBUS_NR_FP64 = 0, ZBUS_NR_MIXED = 1 } zbus_nr_precision;

typedef struct {
  int32_t gmres_restart;      /* Krylov vectors per GMRES cycle, 1 .. 60 (default 30) */
  int32_t gmres_max_restarts; /* GMRES cycles per Newton step, >= 1 (default 4) */
  double gmres_tol;           /* stop a Newton step's GMRES when the preconditioned
                                 residual is below gmres_tol times its start, (0, 1)
                                 (default 1e-6) */
  int32_t precision;          /* zbus_nr_precision (default ZBUS_NR_FP64) */
  int32_t reserved0;
  double reserved[3];
} zbus_nr_opts;

/* Fill *opts with the defaults above. */
void zbus_nr_opts_default(zbus_nr_opts* opts);

/*
 * zbus_nr_network_create -- a transmission grid on the current device.
 *
 *   N          number of buses (>= 2)
 *   nnz        COO entries of the N x N bus admittance matrix (>= 1)
 *   row, col   host int32[nnz]; val_reim host double[2 nnz] (complex, pu;
 *              duplicates summed)
 *   bus_type   host int32[N]: 0 = PQ, 1 = PV, 2 = slack (exactly one; its
 *              angle is the reference 0)
 *   v_set      host double[N]: |V| set-point of PV buses and the slack
 *              (ignored at PQ buses)
 *   eps        diagonal regularisation of B' and B'' (>= 0, e.g. 1e-8)
 *   cuda_stream  stream for the set-up copies; the call returns after them
 *
 * Orders B' + eps I and B'' + eps I by minimum degree and factors them
 * (LU without pivoting).  ZBUS_ERR_SINGULAR if a pivot vanishes,
 * ZBUS_ERR_ARG for invalid input.
 */
zbus_status zbus_nr_network_create(int32_t N, int64_t nnz, const int32_t* row,
                                   const int32_t* col, const double* val_reim,
                                   const int32_t* bus_type, const double* v_set,
                                   double eps, void* cuda_stream, zbus_nr_network* out);

/* Release a grid; NULL is ignored.  No solve of it may still be running. */
void zbus_nr_network_destroy(zbus_nr_network net);

/* Sizes of a grid: angle unknowns, magnitude unknowns, entries of the two
 * preconditioner factors, and the sum of their triangular-solve levels.
 * Any output may be NULL. */
zbus_status zbus_nr_network_info(zbus_nr_network net, int32_t* n_theta, int32_t* n_q,
                                 int64_t* factor_nnz, int32_t* factor_levels);

/*
 * zbus_nr_solve -- Newton-Raphson over B scenarios from the flat start
 * (theta = 0, |V| = 1 at PQ buses, the set-point elsewhere).
 *
 *   P, Q         device double[B][N]: net injections (generation - load, pu);
 *                P of the slack and Q of PV buses and the slack are ignored
 *   tol          converged when max |F_b| <= tol (pu)
 *   max_iter     Newton steps at most (>= 0)
 *   opts         NULL for zbus_nr_opts_default
 *   V_out        device complex [B][N]: the last iterate
 *   iters        device int32[B]: Newton steps taken
 *   converged    device uint8[B]: 1 if max |F_b| <= tol was reached; a
 *                non-finite mismatch stops the scenario unconverged
 *   gmres_iters  device int32[B] or NULL: GMRES iterations (Jacobian-vector
 *                products inside the Krylov cycles) of all Newton steps
 *   cuda_stream  all work is enqueued on this stream
 *
 * Each scenario is solved by one CTA from start to stop (no host round trip
 * per step).  Scratch ((gmres_restart + 6) dim + 9 N doubles per resident
 * CTA, dim = n_theta + n_q; up to eight CTAs per SM) grows on demand with a
 * synchronous allocation.  Device buffers only.  B = 0 is a no-op.  Returns
 * ZBUS_ERR_ARG for a grid whose per-CTA shared work space (N + a few
 * (gmres_restart + 1)^2 doubles) exceeds 227 KB (N above about 27000).  The
 * scratch belongs to the grid: solves of one grid must not overlap on the
 * GPU (other streams or host threads); solves of different grids may.
 */
zbus_status zbus_nr_solve(zbus_nr_network net, int64_t B, const double* P, const double* Q,
                          double tol, int32_t max_iter, const zbus_nr_opts* opts,
                          double* V_out, int32_t* iters, uint8_t* converged,
                          int32_t* gmres_iters, void* cuda_stream);

/*
 * zbus_checked_status -- 1 if this library is the checked build (compiled
 * with -DZBUS_CHECKED, libzbus_checked.so), else 0.  In the checked build
 * every index the kernels read from a table (columns, active lists, tree
 * nodes, maps, permutations, level lists) is tested against its buffer
 * before use; a bad one records a code (0x1nn plain FP64 kernels, 0x2nn
 * tensor-core and tree engine, 0x3nn load gradient, 0x4nn Newton-Raphson,
 * 0x5nn partial-phase maps) and the access is skipped instead of faulting.
 * *word (may be NULL) receives the first code recorded since the last call,
 * 0 if none (always 0 in the normal build), and the codes are cleared.
 * Synchronises the current device.  Project-written: the paper has no
 * counterpart (it stands in for a memory checker on machines where none may
 * run).
 */
int32_t zbus_checked_status(uint32_t* word);

/*
 * zbus_checked_set_wait -- checked build only: the time limit, in
 * nanoseconds, of every wait of the tensor-core pipeline (default 2e9).  0
 * makes a wait that is not complete at its first test give up at once, so a
 * test can make the pipeline give up without a fault: the kernel records
 * ZBUS_ERR_TIMEOUT for zbus_last_device_status, waits (2 s at most) for the
 * MMAs and TMA loads it already issued, frees its tensor memory and ends the
 * sweep loop.  Synchronous.  ZBUS_ERR_UNSUPPORTED in the normal build.
 * Project-written: the paper has no counterpart.
 */
zbus_status zbus_checked_set_wait(uint64_t wait_ns);

/*
 * zbus_probe_fp64_rate -- measure the FP64 fused multiply-add rate of the
 * current device: one launch of 8 blocks per SM x 256 threads, each running
 * eight independent DFMA chains (no memory traffic), after a short warm-up
 * launch, timed with CUDA events on cuda_stream.  *tflops (may be NULL)
 * receives 2 flop per DFMA / the kernel's duration, in TFLOP/s; *ms (may be
 * NULL) the duration.  Synchronous; allocates and frees a few KB on the
 * stream.  The roofline denominator of the FP64 kernels (the plain method's
 * contraction, the mismatch test); project-written, the paper has no
 * counterpart.
 */
zbus_status zbus_probe_fp64_rate(double* tflops, float* ms, void* cuda_stream);

/* Human-readable name of a status code (static storage). */
const char* zbus_status_string(zbus_status s);

/* Message of the last failing call on the calling thread ("" if none). */
const char* zbus_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ZBUS_H */
