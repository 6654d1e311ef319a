/*
 * gribov.h -- C ABI of the B300 Gribov-copy enumerator for compact U(1)
 * lattice Landau gauge in d = 1..4 dimensions.
 *
 * Method (Mehta & Schroeck, arXiv:1403.0555):
 *   links      U_{x,mu} = exp(i phi_{x,mu}), gauge g_x = exp(i theta_x);
 *   functional F(theta) = sum_{x,mu} (1 - cos(phi_{x,mu} + theta_{x+mu} - theta_x))      (Eq. 3)
 *   a Gribov copy is a stationary point of F; the copies counted are those in
 *   the first Gribov region, where the Faddeev-Popov operator (the Hessian of
 *   F in theta) is non-negative apart from its constant zero mode (Section I);
 *   they are found by relaxation (local maximisation of Eq. 4 with K_x of
 *   Eq. 5, checkerboard order) from many random gauge starts (Section III),
 *   stopped when the largest squared lattice divergence is below eps, and
 *   told apart after fixing the global phase theta_{(N,...,N)} = 0 (Section II).
 *
 * Lattice layout used by every array below: V = L^d sites, site index
 * idx(x) = sum_mu x_mu L^mu (x_0 fastest); link (x, mu) at idx(x)*d + mu.
 *
 * Conventions: every entry point returns GC_OK (0) or a negative GC_E* code
 * and then leaves a message for gc_last_error() (per thread).  Host pointers
 * are owned by the caller; all device memory is owned by the library, which
 * allocates it through gc_set_allocator's hooks (cudaMalloc when none are set).
 * The library uses whichever CUDA device is current when an orbit is created.
 */
#ifndef GRIBOV_H
#define GRIBOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define GC_OK 0
#define GC_EINVAL (-1)     /* bad argument (message says which)             */
#define GC_ENOMEM (-2)     /* device or host allocation refused             */
#define GC_ECUDA (-3)      /* a CUDA call failed (message has the CUDA text) */
#define GC_ETIMEDOUT (-4)  /* a bounded device wait ran out                 */
#define GC_ESTATE (-5)     /* call not valid in the orbit's current state   */

/* precision of the relaxation */
#define GC_FP64 0   /* FP64 sweeps, every operation an IEEE-rounded step (no FMA) */
#define GC_MIXED 1  /* FP32 sweeps to eps32, then FP64 polish to eps             */

/* Faddeev-Popov test */
#define GC_FP_AUTO 0     /* FP32 Lanczos screen, FP64 Lanczos near lambda_2 = 0 */
#define GC_FP_LANCZOS 1  /* FP64 Lanczos for every copy                         */
#define GC_FP_DENSE 2    /* FP64 Lanczos, full reorthogonalisation, dim V-1     */
#define GC_FP_NONE 3     /* no test (region reported as -1)                     */

/* FP32-phase kernel: AUTO picks the line-owner kernel where it exists
 * (4^4, 8^3), GENERIC forces the generic team kernel */
#define GC_RELAX_AUTO 0
#define GC_RELAX_GENERIC 1

/* dedup modes (gc_options.dedup_mode) */
#define GC_DEDUP_CONFIG 0   /* distinct canonical configurations (and the F set)   */
#define GC_DEDUP_F8 1       /* the paper's count only (Section III): the set of
                               floor(F/(dV) * 1e8) with the starts reaching each;
                               no configuration table, no first-region test       */

/* per-start status */
#define GC_START_CONVERGED 1
#define GC_START_NOT_CONVERGED 2
#define GC_START_DEDUP_FAILED 3

/* region flag of a distinct copy */
#define GC_REGION_UNTESTED (-1)
#define GC_REGION_OUT 0       /* lambda_2 < -fp_tau: a saddle          */
#define GC_REGION_IN 1        /* lambda_2 > fp_tau: a minimum           */
#define GC_REGION_MARGINAL 2  /* |lambda_2| <= fp_tau                   */

typedef struct gc_orbit_s* gc_orbit;

typedef struct {
  int precision;        /* GC_FP64 or GC_MIXED                                      */
  int check_every;      /* sweeps between residual checks, >= 1                     */
  int max_sweeps;       /* sweep cap per start (rounded up to a multiple of
                           check_every); a start that reaches it is NOT_CONVERGED  */
  double eps32;         /* GC_MIXED: the FP32 phase stops at max div^2 < eps32     */
  double dedup_delta;   /* copies are one when max_x |g'_A - g'_B| <= delta        */
  double fp_tau;        /* marginal band of the Faddeev-Popov test                 */
  int fp_mode;          /* GC_FP_*                                                  */
  int lanczos_k;        /* cap on FP64 Lanczos steps (<= V-1 is used; at least 8L
                           on lattices beyond shared memory)                       */
  uint64_t seed;        /* start generator key word 0 (word 1 is the orbit id)     */
  int keep_per_start;   /* keep the last call's per-start records for fetch_starts */
  int newton_inner;     /* GC_MIXED: cap on FP32 SOR sweeps per Newton polish step */
  int newton_max;       /* GC_MIXED: Newton steps before FP64 relaxation fallback  */
  int batch_starts;     /* starts per device batch, 0 = automatic                  */
  void* stream;         /* cudaStream_t the work is ordered on (NULL = default)    */
  int relax_variant;    /* GC_RELAX_AUTO or GC_RELAX_GENERIC (FP32 phase kernel)    */
  int async;            /* gc_enumerate_batch: return once enqueued (results are
                           complete when opt->stream reaches this point)          */
  int use_graph;        /* gc_enumerate_batch: capture the whole batch as one CUDA
                           graph and launch it (needs a non-default stream)       */
  int autotune;         /* 0 off; 1 tune launch shapes on first use of a (d, L,
                           precision) (results unchanged); 2 also the sweep-unroll
                           depth (mixed precision: sweeps between residual checks,
                           replacing check_every; results move within tolerance) */
  int dedup_mode;       /* GC_DEDUP_CONFIG or GC_DEDUP_F8 (applies per call; the
                           F set is kept in both modes)                           */
} gc_options;

typedef struct {
  uint64_t n_starts;             /* starts relaxed so far (all calls)            */
  uint64_t n_converged;          /* reached eps (FP64 residual)                  */
  uint64_t n_not_converged;
  uint64_t n_dedup_failed;       /* lock wait ran out or copy pool full          */
  uint64_t n_distinct;           /* distinct canonical copies                    */
  uint64_t n_distinct_F8;        /* distinct floor(F/(dV) * 1e8) (Section III)   */
  uint64_t n_in, n_marginal, n_out, n_untested;   /* region flags of copies   */
  uint64_t sweeps_fp32, sweeps_fp64;               /* summed over starts       */
  uint64_t site_updates_fp32, site_updates_fp64;
  uint64_t newton_steps, newton_inner_sweeps, polish_fallbacks, fp64_residual_passes;
  uint64_t fp_tests, fp_tests_fp64, lanczos_steps;
  double ms_relax, ms_polish, ms_dedup, ms_fptest; /* device ms, all calls      */
  uint64_t kernel_launches;      /* kernels the library launched for this orbit */
  uint64_t df_residual_passes;   /* double-float residual passes of the polish   */
  double ms_polish_redo;         /* part of ms_polish: polish_kernel rerunning the
                                    starts the line polish left (4^4); beyond
                                    shared memory, the FP64 sweeps of the starts
                                    the Newton polish left plus the final pass */
  uint64_t polish_redo_starts;   /* starts it reran                              */
  uint64_t lanczos_steps_fp64;   /* part of lanczos_steps taken in FP64 (Lanczos
                                    mode: the FP64 steps after the FP32 seed)   */
  double ms_starts;              /* part of ms_relax before the FP32 sweeps: the
                                    kernel drawing the random starts ahead of
                                    the 4^4 FP32 sweeps; beyond shared memory
                                    (mixed) the FP64 head sweeps from the random
                                    starts; 0 where the sweeps draw their own  */
} gc_stats;

/* Device memory hooks (e.g. a framework's caching allocator).  alloc returns
 * NULL on failure; both are called on the orbit's stream.  Set before creating
 * orbits; NULL hooks restore cudaMalloc / cudaFree. */
typedef void* (*gc_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*gc_free_fn)(void* ptr, void* stream, void* ctx);
int gc_set_allocator(gc_alloc_fn alloc, gc_free_fn free_fn, void* ctx);

/* Defaults: GC_FP64, check_every 1, max_sweeps 100000, eps32 1e-10,
 * dedup_delta 1e-6, fp_tau 1e-9, GC_FP_AUTO, lanczos_k 300, seed 1,
 * keep_per_start 0, newton_inner 320, newton_max 6, batch automatic. */
int gc_options_default(gc_options* opt);

/* Orbit from link angles phi (host, V*d doubles, radians, any range).
 * The library stores (cos phi, sin phi) in FP64 and FP32 (no trigonometry in
 * the sweeps).  orbit_id keys the random starts together with the seed.
 * max_copies sizes the first copy pool (0 = automatic; it grows on demand).
 * d in 1..4, L >= 2.  Lattices whose links and tables fit one CTA's shared
 * memory (e.g. up to 6^4, 14^3, 63^2) take the shared-memory kernels; larger
 * ones, up to V = 65 536 sites with even L and d >= 2 (e.g. 16^4, 40^3,
 * 256^2), take the path for lattices beyond shared memory: hyperplanes of
 * each start streamed from global memory, or held in a cluster's distributed
 * shared memory, with the first-region test by Lanczos in global memory.
 * Anything else is GC_EINVAL. */
int gc_create_orbit(int dim, int L, const double* link_angles, uint64_t orbit_id,
                    size_t max_copies, gc_orbit* out);

/* Relax n_starts new random starts (indices continue across calls, so two
 * calls of n equal one call of 2n), keep the converged ones, deduplicate them
 * into the orbit's table and test each new distinct copy.  omega in (0, 2) is
 * the overrelaxation parameter (1 = the paper's plain relaxation), eps > 0 the
 * stop on max_x div(x)^2.  Returns when the work is complete on opt->stream.
 * GC_ETIMEDOUT: some start's table lock wait ran out (it is counted in
 * n_dedup_failed, everything else is valid). */
int gc_enumerate_copies(gc_orbit o, uint64_t n_starts, double omega, double eps,
                        const gc_options* opt);

/* Many orbits (any mix of d and L) in one call: after a synchronous set-up
 * (copy pools reserved for every start, staging buffers, optional autotuning)
 * each orbit's whole path is enqueued on its own stream of a library pool,
 * forked from and joined back to opt->stream, so the orbits' kernels run
 * concurrently and fill each other's tails.  With opt->use_graph the fork,
 * every kernel and the join are captured as one CUDA graph and launched once.
 * n_starts[i] new starts for orbits[i]; each orbit appears at most once.
 * Per-orbit results are exactly those of gc_enumerate_copies with the same
 * arguments (launch shapes never change a start's arithmetic). */
int gc_enumerate_batch(gc_orbit* orbits, int n_orbits, const uint64_t* n_starts, double omega,
                       double eps, const gc_options* opt);

/* Autotuner: picks warps per CTA of the relaxation, polish and FP-test
 * kernels for o's (d, L) and precision from four pilot runs on a throw-away
 * copy of the orbit; cached per process and used by every later call.  A
 * value is a cap on warps per CTA (16: no cap, the largest shape that fits).
 * The knobs do not change results. */
int gc_autotune(gc_orbit o, int precision, int* r_warps, int* p_warps, int* f_warps);

/* The same with the mode of gc_options.autotune (1 or 2); *check_every gets
 * the tuned sweep-unroll depth in mode 2 with GC_MIXED, else 0. */
int gc_autotune_ex(gc_orbit o, int precision, int mode, int* r_warps, int* p_warps,
                   int* f_warps, int* check_every);

/* Serving with continuous batching and device-side admission.  The server
 * owns a device arena of mem_budget_bytes (0 = half the device's memory,
 * halved until the allocator gives it) and a request loop resident on the
 * GPU: one warp that polls
 * a mailbox in pinned memory, keeps the queue of waiting requests and the
 * arena's region table in device memory, and admits requests in arrival
 * order as soon as a free region fits their device-memory need (links,
 * a copy pool reserved for n_starts copies, one staging batch).  Each
 * admitted request runs on one of `workers` host threads (each on its own
 * stream) with all of its device state carved from its region, so requests
 * that arrive while others run are admitted as memory frees up and their
 * kernels overlap on the GPU.  When it is done, its results move out of the
 * arena (the orbit handed to the caller) and the region goes back to the loop.
 * A request's result does not depend on what else runs.  The loop sleeps
 * between polls and ends after about 0.2 s without work (its state stays on
 * the device; gc_server_state then reports loop_status GC_ETIMEDOUT); the next
 * mail starts it again.
 *   gc_server_submit: GC_ENOMEM if the request alone exceeds the budget.
 *   gc_server_wait:   blocks up to timeout_s (< 0: no limit); GC_ETIMEDOUT if
 *     not finished (the ticket stays valid).  On completion *status is the
 *     request's own result code, *latency_s the time from submission to
 *     completion, and *orbit the finished orbit (NULL on failure; if the
 *     caller passes NULL for orbit, the library destroys it).  The ticket is
 *     then retired.
 *   gc_server_state:  a snapshot of the loop and its admission counters.
 *   gc_server_destroy: finishes submitted requests, stops the loop, frees
 *     orbits nobody collected. */
typedef struct gc_server_s* gc_server;
typedef struct {
  int loop_status;          /* GC_OK, or GC_ETIMEDOUT when the loop's last launch
                               ended on its idle limit                          */
  int loop_running;         /* 1 while a launch of the loop runs                 */
  uint64_t loop_launches;   /* launches of the loop so far                       */
  uint64_t admitted;        /* requests the loop admitted                        */
  uint64_t released;        /* regions mailed back                               */
  uint64_t waiting;         /* requests read by the loop, not yet admitted       */
  uint64_t bytes_in_use;    /* arena bytes of admitted regions                   */
  uint64_t budget_bytes;    /* the arena's size                                  */
  uint32_t regions;         /* entries of the region table (used and free)       */
} gc_server_info;
int gc_server_create(int workers, size_t mem_budget_bytes, const gc_options* opt, gc_server* out);
int gc_server_submit(gc_server s, int dim, int L, const double* link_angles, uint64_t orbit_id,
                     uint64_t n_starts, double omega, double eps, uint64_t* ticket);
int gc_server_wait(gc_server s, uint64_t ticket, double timeout_s, int* status, double* latency_s,
                   gc_orbit* orbit);
int gc_server_state(gc_server s, gc_server_info* out);
int gc_server_destroy(gc_server s);

/* Distinct copies sorted by (F, first_start).  capacity = 0 only sets
 * *n_distinct.  Otherwise the first min(capacity, n) copies are written to
 * every non-NULL array: F[n], theta[n*V] (canonical angles, theta'_{V-1} = 0),
 * first_start[n] (lowest start index reaching the copy), count[n] (starts
 * reaching it), lambda2[n] (NaN when untested), region[n] (GC_REGION_*). */
int gc_fetch_copies(gc_orbit o, size_t capacity, size_t* n_distinct, double* F, double* theta,
                    uint64_t* first_start, uint64_t* count, double* lambda2, int* region);

/* The same fetch, returning once the copies are enqueued.  The call waits
 * for the orbit's earlier work (it reads the number of distinct copies) and
 * orders the copies on the orbit's stream (waiting for that short sort),
 * then enqueues the gathering kernels and the device-to-host copies into the
 * arrays on a separate read-back stream, after the ordering.  The arrays must be page-locked (pinned) for the copies to run
 * asynchronously, and must stay valid and unread until gc_fetch_wait(o)
 * returns; a later fetch of the same orbit, and gc_destroy_orbit, wait for
 * the copies first.  Meanwhile other orbits' work (for example the next
 * batch) can run on the GPU beside the copies.  Errors as gc_fetch_copies. */
int gc_fetch_copies_async(gc_orbit o, size_t capacity, size_t* n_distinct, double* F, double* theta,
                          uint64_t* first_start, uint64_t* count, double* lambda2, int* region);
/* Waits for the copies of the orbit's last gc_fetch_copies_async. */
int gc_fetch_wait(gc_orbit o);

/* Checkpoint / resume: restores into a new orbit (created by gc_create_orbit
 * with the same dimension, size, link angles and orbit id, no starts run
 * yet) the state a run reached, from what gc_fetch_copies (n copies, in any
 * order) and gc_fetch_minima_f8 (n_minima quantised minima and their counts)
 * returned for it.  next_start is the first start index of the next call:
 * the number of starts the run had taken, above every first_start.  Later
 * calls then draw starts next_start, next_start + 1, ... and deduplicate
 * against the restored copies, so the results equal those of the run
 * continued without the break (angles to rounding: the configurations are
 * rebuilt as (cos theta', sin theta')).  The restored copies keep their
 * counts, first starts, lambda_2 and region flags and are not tested again.
 * The orbit's counters (gc_orbit_stats' starts, sweeps and timings) count
 * only the work after the restore.  Host arrays; the call synchronises the
 * orbit's stream.  Errors: GC_ESTATE if the orbit has run starts or holds
 * copies, or belongs to a server; GC_EINVAL for NULL arrays, a first_start
 * at or above next_start, a zero count, a region flag outside -1..2 or a
 * negative F_norm; GC_ENOMEM if the copy pool cannot hold n copies. */
int gc_load_copies(gc_orbit o, size_t n, const double* F, const double* theta, const uint64_t* first_start,
                   const uint64_t* count, const double* lambda2, const int* region, size_t n_minima,
                   const double* F_norm, const uint64_t* minima_count, uint64_t next_start);

/* The paper's set of minima (Section III: minima told apart by F quantised
 * at 1e-8): the distinct keys floor(F/(dV) * 1e8) of every converged start so
 * far, in both dedup modes, in increasing order.  n_minima receives their
 * number; with capacity > 0 the first min(capacity, n) are written: F_norm[i]
 * = key * 1e-8 (the bin's lower edge) and, when count is not NULL, count[i] =
 * the starts whose minimum fell in bin i.  Synchronises with the orbit's
 * stream.  Returns GC_EINVAL for a NULL orbit or n_minima. */
int gc_fetch_minima_f8(gc_orbit o, size_t capacity, size_t* n_minima, double* F_norm, uint64_t* count);

/* Per-start records of the last gc_enumerate_copies call (needs
 * keep_per_start): starts first .. first+n-1 must lie in that call's range.
 * copy_idx is the position in gc_fetch_copies' order, -1 if not converged. */
int gc_fetch_starts(gc_orbit o, uint64_t first, uint64_t n, int* status, int* sweeps,
                    double* F, int64_t* copy_idx);

int gc_orbit_stats(gc_orbit o, gc_stats* out);
int gc_destroy_orbit(gc_orbit o);

/* Allocation-free first-region test.  The paper has no counterpart: this is
 * for callers that must not allocate device memory -- work recorded into a
 * CUDA graph, a service whose device memory budget is fixed up front, or a
 * host that hands the library a fixed arena.  It runs the GC_FP_DENSE test
 * (FP64 Lanczos, full reorthogonalisation, dimension V-1) on n caller-owned
 * copies and allocates nothing: its scratch is one fixed 24 MiB device array
 * that every GPU loading this library holds until the process exits.
 *   d_links    device, V*d (cos phi, sin phi) pairs, link (x, mu) at x*d + mu
 *   d_configs  device, n*V (cos theta, sin theta) pairs, copy i at i*V (any
 *              global phase)
 *   d_lambda2  device out, n doubles: lambda_2 of each copy
 *   d_region   device out, n ints: GC_REGION_IN / _MARGINAL / _OUT (fp_tau)
 * Work is queued on `stream`; outputs are valid once it reaches this point.
 * Limits: n <= 65536 per call and V*V*8 bytes of Lanczos basis must fit the
 * array (V <= about 1700); larger requests fail with GC_EINVAL.  The first
 * call on each device looks up the array's device address; make that first
 * call before any stream capture.  All calls share the one array, so calls
 * whose work overlaps on the GPU (other streams, other host threads) race;
 * order them on one stream. */
int gc_fp_test_static(int dim, int L, const double* d_links, const double* d_configs, uint64_t n,
                      double fp_tau, double* d_lambda2, int* d_region, void* stream);

/* Throughput probe of one arithmetic unit on the current device (the paper
 * has no counterpart: it measures the denominators of the kernels' rooflines
 * on the GPU at hand).  kind: GC_PEAK_FFMA (FP32 FMA), GC_PEAK_FFMA2 (packed
 * f32x2 FMA, counted as two), GC_PEAK_DFMA (FP64 FMA), GC_PEAK_RSQ (the
 * special-function unit's approximate reciprocal square root),
 * GC_PEAK_DFMA_LANE1 (FP64 FMA with one active lane per warp, counted once per
 * warp instruction: equal to GC_PEAK_DFMA / 32 when the pipe's cost does not
 * depend on the active lanes).  Every thread of four 256-thread CTAs per SM
 * runs eight independent chains; the best of three timed launches (after a
 * warm-up) gives *ops_per_s, lane operations per second.  Synchronises `stream` (a cudaStream_t, NULL = default);
 * allocates about 0.6 MB of scratch through the allocator hooks.
 * GC_EINVAL for an unknown kind or a NULL ops_per_s. */
#define GC_PEAK_FFMA 0
#define GC_PEAK_FFMA2 1
#define GC_PEAK_DFMA 2
#define GC_PEAK_RSQ 3
#define GC_PEAK_DFMA_LANE1 4
int gc_peak_probe(int kind, void* stream, double* ops_per_s);

/* Test hook of the copy table's bounded lock wait (the paper has no
 * counterpart; it lets a test drive a device-side wait to its limit without
 * faulting or hanging the GPU).  hold = 1 marks every bucket lock of o's copy
 * table as taken, hold = 0 frees them all; spin_budget is the number of tries
 * a lock wait makes before it gives up (0 restores the default, 2^22).  While
 * the locks are held, a start whose copy is not yet in the table cannot insert
 * it: its wait runs out, the start is marked GC_START_DEDUP_FAILED (counted in
 * n_dedup_failed) and gc_enumerate_copies returns GC_ETIMEDOUT; a start whose
 * copy is already in the table is unaffected (its search takes no lock).
 * Synchronises the orbit's stream.  GC_ESTATE before the orbit's first
 * enumeration (no table yet), GC_EINVAL for a NULL orbit or a negative budget. */
int gc_test_dedup_locks(gc_orbit o, int hold, long long spin_budget);

/* message of the last failing call on this thread ("" if none) */
const char* gc_last_error(void);
/* library version string */
const char* gc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GRIBOV_H */
