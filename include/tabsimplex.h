/*
 * tabsimplex.h -- C ABI of the GB300 (sm_103a) dense full-tableau simplex.
 *
 * The method is the standard full-tableau simplex of arXiv 2211.10979,
 * Section III: maximize c^T x subject to A x <= b, x >= 0 (A is m x n), started
 * from the slack basis of Table I, then per iteration
 *   Step 1  entering column: most negative objective-row coefficient (Dantzig),
 *   Step 2  leaving row: minimum ratio rhs_i / T[i][q] over T[i][q] > 0,
 *   Step 3  pivoting: T[i][j] -= T[i][q] * T[p][j] / T[p][q] for i != p and the
 *           pivot row divided by T[p][q],
 * until no negative coefficient is left (optimal) or column q has no positive
 * entry (unbounded) (Section III, Iterate/Finalization Step).
 *
 * Tableau (Table I): (m + 1) rows x W = n + m + 1 logical columns.  Row 0 is
 * the objective row [-c, 0 | z]; rows 1..m are [A, I_m | b].  The constant z
 * column of Table I is not stored (it never changes).  On the device a handle
 * keeps it row-major with a padded leading dimension, either condensed (the
 * default: the n nonbasic columns and the right-hand side, the basic columns
 * being exact unit vectors; see lp_options.layout) or whole.  Every value,
 * pivot and result is the same in both.  Variable indices are 0-based:
 * 0..n-1 are x_1..x_n, n..n+m-1 are the slacks of constraints 1..m.
 *
 * Threads: calls on one handle are not thread-safe; distinct handles are
 * independent.  Every function that can fail records a message retrievable with
 * lp_last_error() on the calling thread.
 *
 * Device memory comes from the allocator installed with lp_set_allocator()
 * (default: stream-ordered allocation on the handle's stream from a memory
 * pool per device that the library creates and that keeps freed memory for
 * reuse until the process exits).  CUDA events and non-blocking streams that
 * handles no longer need are kept for reuse as well (their creation and
 * destruction serialise concurrent callers in the CUDA runtime).  The pool,
 * the events and the streams belong to the device's primary context:
 * resetting the device (cudaDeviceReset) while the library holds them makes
 * later calls fail with LP_ERR_CUDA.
 */
#ifndef TABSIMPLEX_H
#define TABSIMPLEX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handle: owns the device tableau and all work buffers of one LP. */
typedef struct lp_handle *lp_t;

/* Termination status and error codes.  Non-negative values are outcomes of the
 * iteration (Section III, Iterate/Finalization Step, plus the guards added
 * here); negative values are errors. */
typedef enum {
    LP_OPTIMAL = 0,      /* no objective-row entry below -eps_d                 */
    LP_UNBOUNDED = 1,    /* entering column has no entry above eps_p            */
    LP_ITER_LIMIT = 2,   /* max_iters pivots done, not yet optimal              */
    LP_ERR_NUMERIC = 3,  /* pivot element or minimum ratio not finite           */
    LP_ERR_INVALID = -1, /* bad argument (sizes, NULL, b < 0, non-finite data)  */
    LP_ERR_NOMEM = -2,   /* device allocation failed                            */
    LP_ERR_CUDA = -3,    /* a CUDA runtime call failed                          */
    LP_ERR_TIMEOUT = -4, /* a device-wide barrier wait exceeded its time limit  */
    LP_ERR_STATE = -5,   /* call out of order (e.g. solution before a solve)    */
    LP_PENDING = 100     /* lps_wait: the request has not finished yet          */
} lp_status;

enum { LP_RULE_DANTZIG = 0, LP_RULE_BLAND = 1 };
enum { LP_PATH_AUTO = 0, LP_PATH_PERSISTENT = 1, LP_PATH_MULTILAUNCH = 2,
       LP_PATH_TEAM = 3 /* lp_stats.path of an lp_solve_many solve */,
       LP_PATH_CLUSTER = 4, LP_PATH_HYBRID = 5 };
enum { LP_PREC_FP64 = 0, LP_PREC_FP32 = 1 };

/* Solve options.  Initialise with lp_options_init() and change fields. */
typedef struct {
    int rule;                     /* LP_RULE_DANTZIG (with Bland fallback on
                                     cycling) or LP_RULE_BLAND                  */
    double eps_d;                 /* Step 1: column j may enter iff
                                     T[0][j] < -eps_d (default 1e-9)            */
    double eps_p;                 /* Step 2: row i is eligible iff
                                     T[i][q] > eps_p (default 1e-9)             */
    long long max_iters;          /* pivot cap; < 0 means 50 (m + n)            */
    int k_cyc;                    /* consecutive pivots with minimum ratio <= 0
                                     before switching to Bland's rule until the
                                     next positive-ratio pivot; <= 0 disables
                                     (default 50)                               */
    long long barrier_timeout_ns; /* limit of one device-wide barrier wait
                                     (default 2e9 ns); on expiry the solve ends
                                     with LP_ERR_TIMEOUT                        */
    int path;                     /* LP_PATH_AUTO (default): LP_PATH_CLUSTER
                                     for an FP64 condensed tableau that fits
                                     one thread-block cluster's shared memory
                                     (up to 16 blocks, about 227 KB each: the
                                     whole solve on chip, two cluster barriers
                                     per pivot), else the persistent
                                     cooperative kernel when it can be
                                     launched, else one launch per phase;
                                     LP_PATH_PERSISTENT, LP_PATH_MULTILAUNCH or
                                     LP_PATH_CLUSTER force one of them (the
                                     cluster path refuses, LP_ERR_INVALID, an
                                     LP it cannot hold).  LP_PATH_HYBRID: the
                                     paper's CPU+GPU column split (Section
                                     IV): the persistent kernel on a share
                                     gpu_share of the columns, host threads on
                                     the rest, exchanging the Step 1 and Step
                                     2 results every pivot (FP64, condensed
                                     layout; the same pivots and values)      */
    int skip_zero_columns;        /* full layout only: 1 (default): Step 3
                                     leaves untouched every 32-byte group of
                                     columns whose scaled pivot row entries are
                                     all zero (their update is the identity);
                                     0: update every column                     */
    int threads;                  /* threads per block, 0 = default (256)       */
    int blocks;                   /* grid size cap, 0 = all co-resident blocks
                                     (lp_solve_many: blocks per team)           */
    long long log_capacity;       /* pivots whose (q, p) pair is recorded;
                                     0 = none                                   */
    void *stream;                 /* cudaStream_t to run on; NULL = the
                                     handle's own stream                        */
    int precision;                /* LP_PREC_FP64 (default): double tableau,
                                     results equal the FP64 method step by step.
                                     LP_PREC_FP32: float tableau for every pivot
                                     (half the bytes), then the final basis is
                                     refactorised in FP64 on the GPU (x_B, y
                                     solves, primal/dual/gap checks) and FP64
                                     cleanup pivots run until the checks pass   */
    double eps_d_fp32;            /* eps_d of the float pivots (default 1e-5)   */
    double eps_p_fp32;            /* eps_p of the float pivots (default 1e-6)   */
    double recover_tol;           /* FP64 feasibility tolerance of the checks
                                     (default 1e-9, absolute)                   */
    int cleanup_max;              /* cap on FP64 cleanup pivots (default 1000);
                                     beyond it the solve ends LP_ERR_NUMERIC    */
    int layout;                   /* LP_LAYOUT_CONDENSED (default): the device
                                     keeps the objective row and constraint
                                     rows over the n nonbasic columns plus the
                                     right-hand side ((m+1) x (n+1)); the basic
                                     columns of Table I are exact unit vectors,
                                     so every stored value, pivot and result is
                                     the full tableau's, with half the bytes
                                     at m = n.  LP_LAYOUT_FULL: the Table I
                                     tableau itself ((m+1) x (n+m+1))           */
    double gpu_share;             /* LP_PATH_HYBRID (FP64, condensed): the
                                     fraction theta of the nonbasic column
                                     slots kept on the GPU; host threads hold
                                     the rest (Section IV's CPU/GPU split of
                                     the tableau; default 0.95)                */
    int cpu_threads;              /* LP_PATH_HYBRID: host threads of the CPU
                                     share; 0 = the hardware threads less one,
                                     at least 1 (default 0)                    */
} lp_options;

enum { LP_LAYOUT_CONDENSED = 0, LP_LAYOUT_FULL = 1 };

/* Per-solve measurements (device time from CUDA events on the solve stream). */
typedef struct {
    long long iters;              /* pivots performed                           */
    double build_ms;              /* tableau build (Initialization Step)        */
    double pivot_ms;              /* all pivot kernels (Steps 1-3 + iterate)    */
    long long kernel_launches;    /* kernels launched by the solve              */
    double dense_update_bytes;    /* sum over pivots of 2 (m+1) (n+m+1) s bytes
                                     (the full tableau, read + written)         */
    double update_bytes;          /* sum over pivots of the bytes the pivot
                                     kernels have to move: 64 bytes per row and
                                     32-byte column group Step 3 updates (read +
                                     write), plus Steps 1-2 and the staging     */
    int path;                     /* LP_PATH_PERSISTENT, LP_PATH_MULTILAUNCH or
                                     LP_PATH_TEAM (lp_solve_many)               */
    int grid;                     /* blocks of the pivot kernels (team: the
                                     narrow team size)                          */
    int block;                    /* threads per block                          */
    int ld;                       /* leading dimension of the tableau (elems)   */
    double phase_ms[6];           /* as seen by block 0.  Persistent path:
                                     work time of {ratio test (Steps 1-2),
                                     pivot-row staging, rank-1 update (Step
                                     3)}, then the barrier wait after each of
                                     them.  Cluster path: {Step 2, wait at
                                     the first cluster barrier, cluster
                                     minimum and pivot-row slices, wait at the
                                     second cluster barrier, Step 3, Step 1}   */
    int precision;                /* precision of the solve                     */
    int pivot_status;             /* status at the end of the pivot phase       */
    int k;                        /* FP32 path: structural basic variables      */
    int cleanup_pivots;           /* FP32 path: FP64 cleanup pivots             */
    double recover_ms;            /* FP32 path: FP64 recovery time              */
    double primal_violation;      /* FP32 path: max(0, -min basic value)        */
    double dual_violation;        /* FP32 path: max(0, -min objective-row entry)*/
    double gap;                   /* FP32 path: |c^T x - b^T y|                 */
    int layout;                   /* LP_LAYOUT_CONDENSED or LP_LAYOUT_FULL      */
    double create_copy_ms;        /* lp_create: device time of the host-to-
                                     device copy of A, b, c (0: the handle came
                                     from lp_create_device)                     */
    double create_check_ms;       /* lp_create: device time of the input check
                                     (0 when A, b, c are page-locked: the GPU
                                     reads them over the host link and checks
                                     them in the same pass, counted as copy)   */
    double create_wall_ms;        /* lp_create: host time of the whole call
                                     (allocation, copy, check, synchronisation) */
} lp_stats;

/* Fill *opt with the defaults listed above.  NULL is ignored. */
void lp_options_init(lp_options *opt);

/* Create an LP from HOST arrays (Section III problem statement, Table I):
 * A is m x n row-major, b has m entries, c has n entries, all float64.  The
 * data are copied to the device; the caller keeps ownership of its arrays.
 * When all three are page-locked (cudaHostAlloc, cudaHostRegister) and mapped
 * for the current device, one kernel reads them over the host link and checks
 * them in the same pass; otherwise they are copied with cudaMemcpyAsync and
 * checked on the device.  Returns after the copy and the check completed.
 * Requires m > 0, n > 0, every entry finite and b >= 0 (the slack basis must be
 * feasible: Section III, Initialization Step; no phase I).  Returns NULL on
 * error (see lp_last_error()).  Runs on the current CUDA device. */
lp_t lp_create(int m, int n, const double *A, const double *b, const double *c);

/* Same as lp_create with DEVICE pointers (current device).  The arrays are
 * referenced, not copied: they must stay valid and unchanged until
 * lp_destroy.  `stream` (cudaStream_t, may be NULL for the legacy default
 * stream) is the stream on which the arrays are ready; it becomes the handle's
 * stream.  Validation (finite data, b >= 0) runs on the device. */
lp_t lp_create_device(int m, int n, const double *dA, const double *db,
                      const double *dc, void *stream);

/* Build the tableau from (A, b, c) with the slack basis (Section III,
 * Initialization Step, Table I) and iterate Steps 1-3 (Section III; Section IV
 * Steps 1-4 on one GPU) until termination.  Blocks until the device is done and
 * returns the termination status (>= 0) or an error (< 0).  May be called
 * again: every call starts over from the slack basis.  opt == NULL uses the
 * defaults. */
lp_status lp_solve(lp_t h, const lp_options *opt);

/* Solve `count` LPs at once, each from its slack basis (the method of
 * lp_solve: Section III, Initialization Step and Steps 1-3).  One cooperative
 * launch divides the GPU into teams of opt->blocks thread blocks (default 16)
 * -- and, when some LPs carry more than a team's share of the list's work, up
 * to half of the GPU into wide teams of four times as many blocks that take
 * those LPs first; each team takes the next LP from its list, largest first
 * (then helps with the other list), and iterates on
 * its condensed tableau: block b of the team owns a contiguous range of rows,
 * runs the ratio test on them and updates them, with the scaled pivot row and
 * its rows' multipliers in shared memory; two team barriers per pivot.  Meant
 * for many medium LPs, whose pivots are too small to fill the GPU one at a
 * time.  Every pivot and value equals lp_solve's with the same options.
 *   handles  count distinct handles on the current device (lp_create*)
 *   opt      options as lp_solve (NULL = defaults); layout must be
 *            LP_LAYOUT_CONDENSED, log_capacity 0, threads 0 or 256; blocks =
 *            blocks per team; precision LP_PREC_FP32 adds the FP64 recovery
 *            of each LP after the launch
 *   status   HOST output, count entries: each LP's status as lp_solve returns it
 * An LP whose pivot row and row multipliers do not fit one block's shared
 * memory is solved by lp_solve after the launch.  Afterwards each handle
 * answers lp_get_solution, lp_get_tableau and lp_get_stats as after lp_solve
 * (stats.path = LP_PATH_TEAM, stats.pivot_ms = the whole launch, no pivot
 * log).  Returns LP_OPTIMAL when the call ran (per-LP outcomes in status), or
 * an error (< 0) for invalid arguments or a CUDA failure. */
lp_status lp_solve_many(lp_t *handles, int count, const lp_options *opt, lp_status *status);

/* Read the solution out of the final tableau (Table I layout): x_j is the
 * right-hand side of the row where x_j is basic, else 0 (n entries); y_i is the
 * objective-row entry of the slack column of constraint i (m entries, the dual
 * values); obj is the objective row's right-hand side; basis[i] is the 0-based
 * variable basic in constraint row i+1 (m entries); iters is the number of
 * pivots.  After an LP_PREC_FP32 solve, x, y and obj are the FP64 recovery's
 * values and basis lists the final basic variables in ascending order.  Every
 * output is a HOST pointer and may be NULL.  Returns the status of the last
 * solve, or LP_ERR_STATE before any solve. */
lp_status lp_get_solution(lp_t h, double *x, double *y, double *obj, int *basis,
                          long long *iters);

/* Copy the current tableau to HOST memory T ((m + 1) x (n + m + 1) row-major,
 * float64, without the padding; a float tableau is widened; a condensed
 * tableau is expanded on the device: its slots go to their variables'
 * columns and the basic variables get their unit columns).  Returns
 * LP_ERR_STATE before any solve. */
lp_status lp_get_tableau(lp_t h, double *T);

/* Copy the recorded (q, p) pairs of the last solve (q = entering variable,
 * i.e. its Table I column, p = leaving row in 1..m) to HOST arrays of `cap`
 * entries; *count receives the
 * number of pivots recorded (min(iters, log_capacity)). */
lp_status lp_get_pivot_log(lp_t h, int *q, int *p, long long cap, long long *count);

/* Measurements of the last solve. */
lp_status lp_get_stats(lp_t h, lp_stats *stats);

/* Free the handle and all its device memory.  NULL is ignored. */
void lp_destroy(lp_t h);

/* Message of the last failing call on this thread ("" if none). */
const char *lp_last_error(void);

/* Install the device allocator used by later lp_create* calls (process-wide).
 * alloc(bytes, stream, ctx) returns a device pointer or NULL; free(ptr, bytes,
 * stream, ctx) releases it.  Passing NULL for both restores the default
 * (the library's stream-ordered pool).  Returns 0, or -1 if only one is NULL. */
typedef void *(*lp_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lp_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int lp_set_allocator(lp_alloc_fn alloc_fn, lp_free_fn free_fn, void *ctx);

/* Version string of the library. */
const char *lp_version(void);

/* ------------------------------------------------------------------------
 * Batched solve: many small LPs in one persistent launch (one thread block per
 * LP, the LP's tableau in shared memory).  Every LP is the problem of
 * lp_create and is solved by the same method (Section III, Table I start,
 * Steps 1-3 with the same tie rules), FP64.  Results equal lp_solve's entry
 * for entry.  The block keeps the condensed tableau (the nonbasic columns and
 * the right-hand side; the basic columns of the full tableau are unit
 * vectors): 8 ((m+1) ldc + m + 1 + ldc) + 4 (m + n) bytes (ldc = n + 1 or
 * n + 2, odd), e.g. m = n = 128 needs 134 KB.  In shared memory when it fits
 * the device's opt-in block limit (227 KB on GB300), otherwise in a global
 * workspace slice allocated with the batch (one block per LP either way, so
 * larger LPs are better served by lp_solve_many or lp_solve).  The LPs are
 * grouped in size classes (of which 8, 3, 2 and 1 fit one SM's shared memory
 * side by side), one persistent launch per class.
 * ------------------------------------------------------------------------ */
typedef struct lp_batch *lp_batch_t;

typedef struct {
    int threads;                  /* threads per LP (32, 64, 128, 256, 512);
                                     0 = autotune: each shared-memory size class
                                     times the candidates once per device; the
                                     choice is reused by later solves and
                                     batches on that device                     */
    int rule;                     /* as lp_options                              */
    double eps_d, eps_p;          /* as lp_options (defaults 1e-9)              */
    long long max_iters;          /* per LP; < 0: 50 (m + n)                    */
    int k_cyc;                    /* as lp_options (default 50)                 */
    int use_graph;                /* 1 (default): from the batch's second solve
                                     on, the launches of a solve are captured
                                     once in a CUDA graph and replayed (the
                                     first solve launches them directly)        */
    int keep_tableaux;            /* 1: keep every LP's final tableau for
                                     lp_batch_get_tableau (default 0)           */
    void *stream;                 /* cudaStream_t; NULL = the batch's stream    */
} lp_batch_options;

typedef struct {
    double solve_ms;              /* device time of the last solve              */
    long long total_pivots;       /* pivots of all LPs                          */
    long long kernel_launches;    /* kernels of the last solve (graph nodes)    */
    int buckets;                  /* shared-memory size classes used            */
    int threads[5];               /* threads per LP chosen for each class: four
                                     shared-memory size classes, then the LPs
                                     whose tableau lives in global memory       */
    int lps_per_class[5];
    double tune_ms;               /* time spent autotuning (first solve)        */
    int graph;                    /* 1 if the solve replayed a CUDA graph       */
} lp_batch_stats;

void lp_batch_options_init(lp_batch_options *opt);

/* Create a batch from HOST arrays: LP k has m[k] constraints and n[k]
 * variables; A holds the LPs' constraint matrices back to back (each m[k] x
 * n[k] row-major), b the right-hand sides back to back (sum of m[k]) and c the
 * price vectors back to back (sum of n[k]).  Copied to the device before
 * the call returns (page-locked arrays are read by one kernel over the host
 * link, others copied with cudaMemcpyAsync).  Each LP
 * needs m, n > 0, else NULL (lp_last_error names the LP).  Per-LP input errors
 * found on the device (non-finite data, b < 0) are reported as that LP's
 * status. */
lp_batch_t lp_batch_create(int count, const int *m, const int *n, const double *A,
                           const double *b, const double *c);

/* Same with DEVICE arrays (m, n stay host arrays); the arrays are referenced
 * and must stay valid until lp_batch_destroy; `stream` as lp_create_device. */
lp_batch_t lp_batch_create_device(int count, const int *m, const int *n, const double *dA,
                                  const double *db, const double *dc, void *stream);

/* Solve every LP of the batch (from the slack basis).  Blocks until done.
 * Returns LP_OPTIMAL if the launch succeeded (per-LP outcomes come from
 * lp_batch_get), or an error. */
lp_status lp_batch_solve(lp_batch_t h, const lp_batch_options *opt);

/* Per-LP results to HOST arrays (any may be NULL): status[count], iters[count],
 * obj[count], x packed like c (sum of n[k]), y packed like b (sum of m[k]). */
lp_status lp_batch_get(lp_batch_t h, int *status, long long *iters, double *obj, double *x,
                       double *y);

/* Full final tableau of LP `index` ((m+1) x (n+m+1) row-major, HOST), rebuilt
 * from the kept condensed tableau; needs a solve with keep_tableaux = 1. */
lp_status lp_batch_get_tableau(lp_batch_t h, int index, double *T);

lp_status lp_batch_get_stats(lp_batch_t h, lp_batch_stats *stats);

/* Free the batch (NULL is ignored). */
void lp_batch_destroy(lp_batch_t h);

/* ------------------------------------------------------------------------
 * Request server with continuous batching.  Requests (one LP each) enter a
 * FIFO queue; a pool of worker threads, each with its own CUDA stream, admits
 * them in arrival order while the device-memory budget allows.  LPs up to a
 * size (shared-memory fit, or batch_max_bytes) are taken together -- every such
 * request waiting at that moment, up to batch_max -- and solved as one
 * micro-batch (FP64, results equal lp_solve's); the others are solved in
 * waves by lp_solve_many with the given precision (default FP32 tableau + FP64
 * recovery): every such request waiting when a wave is formed joins it; the
 * next wave is formed while the current one's team launch runs, and the
 * finished wave's recovery and read-out overlap the next launch (or, with
 * team_blocks < 0, one per worker by lp_create / lp_solve on a share of the
 * GPU's blocks).  By default (continuous = 1) there are no waves: one team
 * launch stays resident while requests keep coming, each admitted large
 * request is appended to its job list at once and taken by the next free
 * team, and each result is finished (FP64 recovery, read-out) as soon as its
 * own team is done.  Requests arriving while others are on the GPU are
 * admitted as workers and memory free up, and their work overlaps on the
 * device.  The paper has no serving layer; every solve inside is the method of
 * lp_solve.
 * ------------------------------------------------------------------------ */
typedef struct lp_server *lps_t;

typedef struct {
    long long budget_bytes;       /* device bytes admitted requests may hold
                                     (tableau, inputs, work; default 64 GiB)    */
    int workers;                  /* concurrent solves (default 8)              */
    int precision;                /* single-LP lane (default LP_PREC_FP32)      */
    int batch_small;              /* 1 (default): micro-batch the small LPs     */
    int batch_max;                /* max LPs per micro-batch (default 1024)     */
    int small_max_dim;            /* > 0: micro-batch only LPs with m, n <= this;
                                     0 (default): every LP that fits the
                                     batched solver's shared memory             */
    int blocks_per_lp;            /* grid cap of a single-lane solve; 0
                                     (default): 4 x SMs / workers, at least 16  */
    long long batch_max_bytes;    /* > 0: LPs whose condensed tableau (8 (m+1)
                                     (n+2) bytes) is at most this also go
                                     through the micro-batches, solved from
                                     global memory one block per LP (pays off
                                     only when many such LPs wait together);
                                     0 (default): shared-memory LPs only        */
    int path;                     /* lp_options.path of the single-lane solves;
                                     default LP_PATH_MULTILAUNCH, whose kernels
                                     overlap with other workers' solves (the
                                     cooperative launches of the persistent
                                     path largely run one at a time)            */
    int team_blocks;              /* >= 0 (default 0: lp_solve_many's default
                                     team of 16 blocks): the requests too
                                     large for the micro-batches are solved in
                                     waves by lp_solve_many with teams of this
                                     many blocks -- every such request waiting
                                     when a wave starts joins it, one wave at a
                                     time; < 0: one per worker by lp_solve     */
    int continuous;               /* 1 (default, with team_blocks >= 0): the
                                     large requests go to one continuous team
                                     launch instead of waves: each is taken by
                                     the next team that finishes an LP as soon
                                     as it is admitted, and its result is
                                     returned as soon as its own team is done
                                     (the launch ends when idle and restarts
                                     with the next request); 0: waves         */
} lps_options;

typedef struct {
    long long submitted, completed;
    double wall_s;                /* first submit to last completion            */
    double lat_p50_ms, lat_p99_ms, lat_mean_ms, lat_max_ms;   /* submit -> done */
    double queue_p50_ms, queue_p99_ms;                        /* submit -> admit*/
    long long batches, batched_lps;
    long long peak_bytes;         /* largest admitted total                     */
    long long waves, wave_lps;    /* lp_solve_many waves and the LPs in them   */
    double wave_ms;               /* wall time of the waves (create, solve,
                                     recovery, read-out), summed                */
    double wave_kernel_ms;        /* device time of their team launches, summed */
    double wave_create_ms;        /* of wave_ms: handle creation               */
    double wave_wait_ms;          /* of wave_ms: waiting for the launch token  */
    double wave_launch_ms;        /* of wave_ms: set-up and team launch (host) */
    /* where a request's latency goes (every completed request):              */
    double wait_p50_ms, wait_p99_ms;  /* admitted -> its solve's launch starts
                                         (a wave waits for the previous one)   */
    double run_p50_ms, run_p99_ms;    /* launch -> its kernel completes (a
                                         wave's whole team launch)             */
    double post_p50_ms, post_p99_ms;  /* kernel done -> result stored (FP64
                                         recovery, read-out)                   */
    long long lane_lps;           /* requests solved by the continuous launch  */
    long long lane_launches;      /* continuous team launches started          */
} lps_stats;

void lps_options_init(lps_options *opt);

/* Start a server on the current device (worker threads start at once).
 * NULL opt = defaults.  Returns NULL on error. */
lps_t lps_open(const lps_options *opt);

/* Submit an LP from HOST arrays (copied before return).  Returns a ticket
 * (>= 0) or -1 on error (bad sizes, larger than the budget, closing). */
long long lps_submit(lps_t sv, int m, int n, const double *A, const double *b, const double *c);

/* Submit an LP whose arrays are on the device (referenced: they must stay
 * valid and unchanged until the request finishes; their contents must be
 * complete when this is called). */
long long lps_submit_device(lps_t sv, int m, int n, const double *dA, const double *db,
                            const double *dc);

/* Wait for a request: its status once finished, or LP_PENDING after
 * timeout_s seconds (timeout_s < 0: no limit). */
int lps_wait(lps_t sv, long long ticket, double timeout_s);

/* Result of a finished request to HOST arrays (any may be NULL): x (n), y (m),
 * objective, pivots; times[3] = submit, admit, done (seconds of a monotonic
 * clock).  Returns the request's status, LP_ERR_STATE if unfinished. */
lp_status lps_result(lps_t sv, long long ticket, double *x, double *y, double *obj,
                     long long *iters, double *times);

/* Forget a finished request (frees its stored result). */
lp_status lps_release(lps_t sv, long long ticket);

lp_status lps_get_stats(lps_t sv, lps_stats *stats);

/* Message of the latest failed solve on any worker ("" if none); valid until
 * the calling thread's next call. */
const char *lps_last_error(lps_t sv);

/* Finish every queued request, stop the workers, free the server. */
void lps_close(lps_t sv);

/* Seeded synthetic LP written on the device (inputs for tests and benchmarks,
 * not part of the method): the dense generator A_ij = 1 + 9u,
 * b_i = 100 + 900u, c_j = 1 + 9u with u from the counter-based SplitMix64
 * stream of `seed` (draws in the order A row-major, b, c), identical to the
 * Python generator lpgen.dense_lp.  dA (m x n), db (m), dc (n) are device
 * arrays; runs on `stream`. */
lp_status lp_generate_dense(int m, int n, unsigned long long seed, double *dA, double *db,
                            double *dc, void *stream);

/* Measurement helper, not part of the method: the device's FP64 fused
 * multiply-add rate, the ceiling of kernels bound by the FP64 pipe (the
 * batched solver).  One launch of `blocks` x `threads` threads (threads a
 * multiple of 32, at most 1024), each running 8 independent chains of
 * `iters` dependent fma(a, x, y) on the current device, on `stream`
 * (cudaStream_t, NULL = legacy default stream).  Blocks until done; *ms_out
 * receives the launch's CUDA-event time and *fma_per_s_out the rate
 * (blocks x threads x 8 x iters / time), both HOST pointers, may be NULL.
 * Allocates blocks x threads doubles of device memory for the chains' results
 * for the duration of the call. */
lp_status lp_measure_fp64_fma_rate(int blocks, int threads, long long iters, void *stream,
                                   double *ms_out, double *fma_per_s_out);

/* Measurement helper, not part of the method: how the FP64 pipe charges a
 * warp instruction.  Same launch as above, but only `lanes` (1..32) lanes of
 * each warp run the chains, of op 0 = fma(a, x, y) or op 1 = IEEE division
 * y / a.  *warp_ops_per_s_out receives warp instructions (chain steps of a
 * warp) per second, whatever the active lanes.  HOST outputs, may be NULL. */
lp_status lp_measure_fp64_op_rate(int op, int lanes, int blocks, int threads, long long iters,
                                  void *stream, double *ms_out, double *warp_ops_per_s_out);

/* Solve without allocating any device memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * themselves or let the library do it -- for example a plugin running inside
 * a host application whose own memory pool has reserved the GPU's memory, or a
 * latency-sensitive loop that must not call cudaMalloc/cudaFree, which can
 * block on or synchronise with other work on the device.
 *
 * It takes the same pivots and gives the same results as lp_create_device
 * followed by lp_solve with the same options, with every buffer supplied by
 * the caller and the work buffers (pivot column, scaled pivot row, reduction
 * partials, status and barrier words) taken from one fixed array that the
 * library holds in device global memory: LP_NOALLOC_SCRATCH_BYTES (2 MiB) on
 * every GPU that loads the library, kept until the process exits.
 *   dA, db, dc  device inputs (m x n row-major, m, n float64), read only;
 *               every entry finite and b >= 0, else LP_ERR_INVALID
 *   dT          device output, (m + 1) x ld float64, 32-byte aligned; receives
 *               the final tableau with every column, basic ones included (rows:
 *               objective, then constraints 1..m; columns: x_1..x_n, the m
 *               slacks, the right-hand side at n + m, zeros after)
 *   ld          leading dimension of dT in elements: >= n + m + 1, multiple of 4
 *   dbasis      device output, m ints: variable basic in constraint row i + 1
 *   opt         options as for lp_solve (NULL = defaults); opt->stream is the
 *               stream used; log_capacity must be 0 and blocks <= 1024
 *   iters       host output (may be NULL): pivots performed
 * opt->layout is ignored: dT always holds every column, as described above.
 * The work buffers need 8 (m + 1) + 9 ld + 32 ceil(ld / 128) + 32 * 1024 bytes
 * plus about 1.5 KiB of alignment and state, at most LP_NOALLOC_SCRATCH_BYTES
 * (about m + ld <= 2.2e5, e.g. m = n = 70000); larger sizes return LP_ERR_INVALID
 * before any device work, with the sizes in lp_last_error().
 * Every call on a device uses the same array and leaves its contents behind
 * (each call resets what must start from zero), so calls whose GPU work
 * overlaps -- concurrent streams or host threads -- race: serialise them.
 * Blocks until the device is done (it reads status words back), so it cannot
 * be recorded into a CUDA graph: on a stream that is being captured it
 * returns LP_ERR_STATE without any device work.  Returns the termination
 * status (>= 0) or an error (< 0). */
#define LP_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u)
lp_status lp_solve_noalloc(int m, int n, const double *dA, const double *db,
                           const double *dc, double *dT, long long ld,
                           int *dbasis, const lp_options *opt, long long *iters);

#ifdef __cplusplus
}
#endif

#endif /* TABSIMPLEX_H */
