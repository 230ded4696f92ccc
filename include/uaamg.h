/*
 * uaamg.h -- C ABI of the GB300 (sm_103a) unsmoothed-aggregation AMG library.
 *
 * The library solves A u = f (Eq. 2.1) for a weighted graph Laplacian A (Section 2):
 * symmetric, a_ij = -w_ij <= 0 off the diagonal, a_ii = sum_j w_ij + wD_i, positive definite
 * because a Dirichlet set S is non-empty on every connected component.
 *
 *   setup (Algorithm 1, setup phase): per level, priorities (Eq. 3.2), parallel aggregation
 *     passes (Algorithm 2), coarse numbering by ascending root (Section 5.1), coarse
 *     operator by aggregate sums (Eq. 2.4), l1-Jacobi data (Section 4.1), and the dense
 *     FP64 inverse of the coarsest matrix (symmetric Gauss-Jordan sweep).
 *   solve (Algorithm 1, solve phase, with the K-cycle of Section 4.3 as preconditioner of
 *     a flexible conjugate gradient, Sections 1 and 4.4): l1-Jacobi smoothing fused into
 *     CSR SpMV, aggregate-sum restriction and piecewise-constant prolongation
 *     (Section 4.2), two flexible-CG steps per coarse level.
 *
 * Every compute step runs in this library's CUDA kernels on the caller's stream.  There is
 * no CPU fallback: without a usable CUDA device every call that computes returns
 * UAAMG_ERR_CUDA.
 *
 * Conventions
 *  - Indices are 0-based int32.  CSR: rowptr[n+1], col[nnz] strictly ascending within each
 *    row, the diagonal stored, val[nnz] float64.  The pattern and values must be
 *    symmetric; the diagonal must be positive.
 *  - Pointers are host or device addresses as stated per argument.  The library never
 *    keeps a caller pointer after a call returns.
 *  - Every function returns a status code (UAAMG_OK = 0) and never throws.  On an error
 *    the output arguments are unspecified unless stated.
 *  - A handle is used by one host thread at a time and runs all its work on the stream
 *    given at setup; different handles may run concurrently on different streams.
 */
#ifndef UAAMG_H
#define UAAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define UAAMG_OK 0
#define UAAMG_ERR_INVALID_ARG 1   /* null pointer, out-of-range parameter */
#define UAAMG_ERR_BAD_CSR 2       /* malformed, unsorted, asymmetric, non-finite, bad diag */
#define UAAMG_ERR_NOT_SPD 3       /* a pivot <= 0 while inverting the coarsest matrix */
#define UAAMG_ERR_NO_CONVERGENCE 4 /* max_iter reached; iters/relres/x are still filled */
#define UAAMG_ERR_OOM 5           /* device allocation failed */
#define UAAMG_ERR_BUDGET 6        /* the library-wide device-memory budget would be exceeded */
#define UAAMG_ERR_CUDA 7          /* a CUDA runtime call failed (no device, launch error) */
#define UAAMG_ERR_TIMEOUT 8       /* a bounded device-side wait gave up */
#define UAAMG_ERR_UNSUPPORTED 9   /* a size beyond this build's limits */
#define UAAMG_ERR_CANCELLED 10    /* a queued solve-service request was cancelled */

/* ---- parameters --------------------------------------------------------------------- */
#define UAAMG_FP64 0  /* K-cycle, hierarchy and outer iteration in FP64 */
#define UAAMG_MIXED 1 /* FP32 hierarchy and K-cycle inside the FP64 outer iteration */

#define UAAMG_PASS_SINGLE_ROUND 1 /* Algorithm 2 as printed: one round of local maxima per pass */
#define UAAMG_PASS_MAXIMAL 0      /* a maximal distance-2 independent set per pass (Section 3.1) */

typedef struct uaamg_csr {
    int32_t n;             /* rows = columns, >= 1 */
    int32_t nnz;           /* stored entries, rowptr[n] */
    const int32_t* rowptr; /* [n+1] */
    const int32_t* col;    /* [nnz] */
    const double* val;     /* [nnz] */
    int32_t on_device;     /* 1: the three arrays are device pointers, 0: host pointers */
} uaamg_csr;

typedef struct uaamg_params {
    int32_t coarse_size;  /* coarsen while n_l > coarse_size (Algorithm 1 "n_0"); default 64 */
    int32_t max_levels;   /* at most this many levels, finest included (Algorithm 1 "L"); 25 */
    int32_t max_agg_size; /* t of Section 3.3: 0 = unbounded, else >= 2; default 5 */
    int32_t pass_mode;    /* UAAMG_PASS_SINGLE_ROUND (default) or UAAMG_PASS_MAXIMAL */
    uint64_t seed;        /* seed of the hashed priority vector (Eq. 3.2); default 0x5EED */
    int32_t pre, post;    /* l1-Jacobi sweeps before / after the coarse correction; 1, 1 */
    int32_t kcycle_inner; /* flexible-CG steps per coarse level, 1 or 2; default 2 */
    double kcycle_tau;    /* > 0: skip the second step when |rho~| <= tau |rho|; default 0 */
    int32_t precision;    /* UAAMG_MIXED (default) or UAAMG_FP64 */
    int32_t max_iter;     /* outer iterations; default 200 */
    int32_t use_graphs;   /* 1 (default): run the outer iterations as one CUDA graph whose
                             while node repeats an iteration until the device-side stopping
                             test passes; 0: launch every kernel from the host */
    int32_t profile_class; /* UAAMG_KCLASS_* to time from setup on (0 = none, default) */
    int32_t agg_repeat;   /* 1 (default): one aggregation per level; 2: aggregate the coarse
                             graph once more before forming the level (Section 3.3) */
    double kcycle_ratio;  /* > 0: coarse level m takes its second flexible-CG step only when
                             n_{m-1} / n_m >= kcycle_ratio; default 0 (always two steps) */
    double min_coarsening; /* > 0: a level of at most 1024 unknowns whose aggregation would
                              shrink it by less than this factor becomes the coarsest; 0 */
    double jacobi_omega;  /* 0 (default): l1-Jacobi smoother; > 0: damped Jacobi
                             x += omega D^{-1} (b - A x) (Section 4.1) */
    int32_t tma_rows;     /* levels with at least this many rows run their SpMV-based kernels
                             as persistent blocks that stream the matrix into shared memory
                             with TMA bulk copies, one thread per row (0 = never); default
                             131072.  Changes no vector entry; fused inner products are summed
                             in another fixed order. */
    int32_t sell_rows;    /* levels (except the coarsest) with at least this many rows also
                             keep a sliced ELLPACK copy (slices of 32 rows, column-major;
                             Section 4.4) that their row kernels read instead of the CSR;
                             skipped where it would pad the entries by more than 25% or a row
                             exceeds 65535 entries (0 = never).  Changes no vector entry. */
    int32_t fuse_below;   /* coarse levels with at most this many unknowns run their K-cycle
                             in one fused single-block kernel (pre = post = 1 only); 0 = off
                             (default: on GB300 one block is slower than launching) */
    int32_t sra_rounds;   /* 0 (default) .. 64: rounds of subgraph reshaping (Section 3.2,
                             Algorithm 3) applied to each level's aggregation before its coarse
                             operator is formed (the first stage when agg_repeat = 2).  A round
                             matches neighbouring aggregates in pairs whose union has at most 16
                             vertices (mutual choice of a seeded hashed pair weight) and splits
                             every pair's union into the two connected halves of sizes
                             floor(n/2) and ceil(n/2) that maximise |T(V_c)|_A^2 on the union's
                             local graph Laplacian (l1-Jacobi smoother).  Energies within a
                             relative 1e-9 count as equal (the split whose mask of the union's
                             ascending vertices is smallest wins).  A pair without such a split
                             stays as it is.  The number of aggregates does not change. */
    int32_t restrict_fuse_below; /* levels with at most this many unknowns (on the row-block
                                    kernels, one pre-sweep) run their first sweep and the
                                    restriction in one launch, a warp per aggregate; 0 = never
                                    (default: on GB300 the two launches are faster except on
                                    hierarchies of a few thousand unknowns) */
    int32_t autotune;     /* 1: at the end of setup, time the SpMV-based kernels of a visit of
                             each level of at least 32768 unknowns (first sweep, prolongation
                             sweep, SpMV with two inner products; on level 0 also the FP64
                             outer SpMV) with the row-block kernel at 256, 128, 64 and 32 rows
                             per block, the per-warp TMA kernel and the sliced ELLPACK kernel,
                             and keep the fastest for the level (remembered per level shape for
                             the process); 0 (default): the size thresholds tma_rows and
                             sell_rows decide.  Changes the rounding of row sums only (the
                             lanes a row is split into). */
    int32_t cluster_below; /* coarse levels with at most this many unknowns (and at most 65536)
                              run their K-cycle in one launch on one thread-block cluster
                              (pre = post = 1 only): 16 blocks (8 where the device does not
                              run 16) that hold the levels' vectors and matrices in shared
                              memory, replicate the vectors other blocks gather through
                              distributed shared memory and synchronise by cluster barriers.
                              The tail starts at the first such level whose data fit in the
                              cluster's shared memory, else lower.  Default 8192; 0 = off.
                              Takes precedence over fuse_below.  Changes the rounding of the
                              K-cycle's inner products (FP32 pairs in mixed precision) and of
                              row sums split across lanes. */
    int64_t wait_limit_ns; /* limit of every bounded device-side wait of this handle: a grid
                              barrier of a cooperative kernel, a wait for a bulk copy into
                              shared memory (measured in SM clock cycles, about 2 per ns).
                              A wait that runs out makes the call return UAAMG_ERR_TIMEOUT and
                              leaves the device usable.  0 (default): 2 s per barrier, 2^31
                              cycles per copy wait. */
} uaamg_params;

typedef struct uaamg_handle uaamg_handle;

/* Fills *p with the defaults listed above. */
void uaamg_default_params(uaamg_params* p);

/*
 * Setup phase of Algorithm 1 for the matrix A on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  The CSR is validated on the device (UAAMG_ERR_BAD_CSR), copied
 * into handle-owned device memory, and the hierarchy is built: levels 0 (finest) .. L-1
 * (coarsest, n <= 1024 or UAAMG_ERR_UNSUPPORTED).  The caller's arrays may be freed or
 * reused when the call returns.  The call synchronises `stream` a few times per level to
 * learn level sizes.  On success *out owns all device memory of the hierarchy until
 * uaamg_free; on failure *out is NULL.
 */
int uaamg_setup(const uaamg_csr* A, const uaamg_params* p, void* stream, uaamg_handle** out);

/*
 * Solves A x = b by flexible CG preconditioned with the K-cycle until
 * |b - A x|_2 <= tol |b|_2 for the recomputed FP64 residual, or max_iter iterations.
 * b[n] and x[n] are float64, host or device pointers (detected per call).  use_guess != 0
 * takes the initial x from x, else x0 = 0.  On return x holds the last iterate, *iters the
 * outer iteration count and *relres the final relative residual (both filled also for
 * UAAMG_ERR_NO_CONVERGENCE).  With use_graphs the iterations run on the device until the
 * recursive residual passes the test, and the call synchronises the handle's stream a few
 * times per solve (setup of the residual, that loop, the confirming FP64 residual); without
 * it, or while a kernel class is profiled, it synchronises once per outer iteration.
 */
int uaamg_solve(uaamg_handle* h, const double* b, double* x, double tol, int32_t use_guess,
                int32_t* iters, double* relres);

/*
 * Solves A X = B for nrhs right-hand sides at once (1 <= nrhs <= 32), each column by the
 * same algorithm as uaamg_solve from x0 = 0, with its own K-cycle coefficients, its own
 * outer iteration and its own stopping test; every level's matrix is read once per sweep
 * for all columns.  B and X are float64 arrays of n * nrhs in row-major [n][nrhs] order (the
 * nrhs values of row i are contiguous), host or device pointers.  iters[nrhs] and
 * relres[nrhs] (host) receive each column's outer iteration count and final relative
 * residual of b - A x.  Returns UAAMG_OK when every column converged, else
 * UAAMG_ERR_NO_CONVERGENCE with all outputs filled; UAAMG_ERR_UNSUPPORTED for nrhs > 32 or a
 * handle set up with pre != 1 or post != 1.  Workspace for nrhs columns is allocated on the
 * first call with that many columns and kept by the handle.
 */
int uaamg_solve_many(uaamg_handle* h, int32_t nrhs, const double* B, double* X, double tol,
                     int32_t* iters, double* relres);

/*
 * Solves nsys independent systems together, each with its own hierarchy (a handle from
 * uaamg_setup, all on one device and in one precision, pre = post = 1) and its own nrhs[s]
 * right-hand sides (1 <= nrhs[s] <= 32).  Every column of every system runs the same
 * algorithm as uaamg_solve from x0 = 0, with its own K-cycle coefficients, outer iteration
 * and stopping test (|b - A x|_2 <= tol |b|_2, confirmed on the recomputed FP64 residual).
 * The systems' K-cycles advance together, level step by level step: each step is one launch
 * over every system that takes it (their levels' rows split into tiles), so the launches of
 * an outer iteration do not grow with the number of systems.  A system's result does not
 * depend on which other systems share the call: its tiles, and the order of its inner
 * products, are a function of its own level sizes and nrhs[s] only.
 *   B[s], X[s]: float64 [n_s][nrhs[s]] row-major (the columns of row i contiguous), host or
 *     device pointers; X[s] receives the solutions.
 *   iters, relres (host): one entry per column, systems in order (nrhs[0] entries for
 *     system 0, then system 1, ...): outer iterations and the final relative residual.
 * Returns UAAMG_OK when every column converged within its handle's max_iter, else
 * UAAMG_ERR_NO_CONVERGENCE with all outputs filled; UAAMG_ERR_INVALID_ARG for a repeated
 * or null handle or mixed precisions or devices; UAAMG_ERR_UNSUPPORTED for nrhs outside
 * 1..32, pre/post != 1, or K-cycles whose union needs more than 65536 launches per outer
 * iteration (two flexible-CG steps on many levels make the cycle exponential in depth).  Runs on a stream of its own, ordered after `stream` and after
 * each handle's stream (and they after it); it synchronises once per outer iteration.
 * Each handle keeps a workspace of nrhs[s] columns (as uaamg_solve_many); a handle is used
 * by this call alone while it runs.  The paper has no batched solve: this is the serving
 * extension of its K-cycle (Section 4.3) to many systems at once.
 */
int uaamg_solve_batch(uaamg_handle* const* handles, int32_t nsys, const int32_t* nrhs,
                      const double* const* B, double* const* X, double tol, int32_t* iters,
                      double* relres, void* stream);

/*
 * uaamg_setup(A[s], p[s], stream) for nsys matrices (p = NULL: defaults for all), run on
 * `threads` host threads so that the setups of different matrices (each on its handle's own
 * stream) overlap on the device.  out[s] receives system s's handle, whose caller's stream
 * is `stream`.  All or nothing: on the first failing status every handle made is freed,
 * out[] is all NULL and that status is returned.
 */
int uaamg_setup_batch(int32_t nsys, const uaamg_csr* A, const uaamg_params* p, int32_t threads,
                      void* stream, uaamg_handle** out);

/* Releases every device allocation of the handle (stream-ordered on its stream). */
void uaamg_free(uaamg_handle* h);

/* ---- introspection, used by the parity tests ---------------------------------------- */
int uaamg_num_levels(const uaamg_handle* h, int32_t* nlev);
/* n, nnz and the number of aggregation passes of level l (passes = 0 on the coarsest). */
int uaamg_level_info(const uaamg_handle* h, int32_t l, int32_t* n, int32_t* nnz,
                     int32_t* passes);
/* Host copies: agg[n_l] (column of P holding each row, l < L-1), and the level matrix. */
int uaamg_get_aggregates(const uaamg_handle* h, int32_t l, int32_t* agg);
int uaamg_get_level_csr(const uaamg_handle* h, int32_t l, int32_t* rowptr, int32_t* col,
                        double* val);
/* Host copies of the priority vector (Eq. 3.2) of level l and of the pass in which each
 * vertex was aggregated (l < L-1). */
int uaamg_get_priorities(const uaamg_handle* h, int32_t l, uint64_t* P);
int uaamg_get_pass_of(const uaamg_handle* h, int32_t l, int32_t* pass_of);
/* The kernel family level l's SpMV-based kernels run (*path: 0 row-block with *rows rows
 * per block, 1 per-warp TMA, 2 sliced ELLPACK) and the autotuner's timings of one visit's
 * kernels in microseconds (us[6]: row-block 256, 128, 64, 32, TMA, ELLPACK; -1 where not
 * timed, all -1 when the level was not tuned). */
int uaamg_level_kernel(const uaamg_handle* h, int32_t l, int32_t* path, int32_t* rows,
                       double* us);
/* Host copy of the FP64 l1-Jacobi diagonal Minv_i = 1 / (a_ii + sum_{j!=i} |a_ij|). */
int uaamg_get_minv(const uaamg_handle* h, int32_t l, double* minv);
/* Applies the level-l preconditioner B_l (l < L-1) or the level-m K-cycle K_m (m >= 1) to a
 * host vector in the handle's precision; out and in are host float64 arrays of n_l. */
int uaamg_apply_B(uaamg_handle* h, int32_t l, const double* in, double* out);
int uaamg_apply_K(uaamg_handle* h, int32_t m, const double* in, double* out);
/* Relative residual |b - A x| / |b| after each outer iteration of the last solve
 * (hist[0] = initial); *count receives min(cap, iterations + 1). */
int uaamg_residual_history(const uaamg_handle* h, double* hist, int32_t cap, int32_t* count);

/* ---- measurement -------------------------------------------------------------------- */
typedef struct uaamg_stats {
    double setup_ms;      /* device time of the last setup (CUDA events) */
    double solve_ms;      /* device time of the last solve */
    int64_t launches;     /* kernels launched by this handle (graph nodes counted per replay) */
    int64_t graph_nodes;  /* kernel nodes of one outer iteration in the last graph built */
    double opc;           /* operator complexity sum_l nnz_l / nnz_0 */
    double grid_complexity;
    uint64_t device_bytes; /* device memory the handle holds now (hierarchy and workspace) */
    int32_t tail_level;    /* first level of the fused small-level K-cycle kernel, 0 = none */
    int32_t tail_blocks;   /* its thread blocks: the cluster size, 1 for the one-block kernel */
} uaamg_stats;
int uaamg_get_stats(const uaamg_handle* h, uaamg_stats* s);

/*
 * Kernel timing hooks.  When enabled (params.profile_class at setup for the setup classes,
 * or uaamg_set_profiling before the first solve of a handle), level-0 launches of the
 * selected kernel class are bracketed by CUDA events on the launching stream and the
 * durations accumulate: every such launch of the setup, and for the solve classes the
 * launches of the first three outer iterations of each solve, which then run launch by
 * launch (the remaining iterations run in the device-side loop, which holds no events).
 */
#define UAAMG_KCLASS_SMOOTH0 1  /* level-0 first l1-Jacobi sweep + residual (fused SpMV) */
#define UAAMG_KCLASS_SPMV64 2   /* level-0 FP64 SpMV + dot kernel of the outer iteration */
#define UAAMG_KCLASS_PAA 3      /* the aggregation kernel of setup level 0 */
#define UAAMG_KCLASS_COARSE 4   /* the coarse-operator assembly kernel of setup level 0 */
#define UAAMG_KCLASS_SRA 5      /* the pair kernel of subgraph reshaping on setup level 0; its
                                   "bytes" per launch are FP64 operations per launch */
int uaamg_set_profiling(uaamg_handle* h, int32_t kclass);
/* launches, total ms, and algorithmic bytes moved per launch of the profiled class (for
 * UAAMG_KCLASS_SRA: algorithmic FP64 operations per launch, counted by the kernel) */
int uaamg_get_profile(const uaamg_handle* h, int64_t* launches, double* total_ms,
                      double* bytes_per_launch);

/* The device's FP64 fused multiply-add rate (FMA per second, an FMA being two floating-point
 * operations), measured with CUDA events over `chains` (1 or 8) independent FMA recurrences
 * per thread on a grid of resident blocks on every SM (1: latency-bound, 8: the pipe's
 * throughput).  The denominator of the FP64 roofline; runs on the legacy default stream. */
int uaamg_measure_fp64_fma(int32_t chains, double* fma_per_s);

/* Total kernels launched by this library in this process (all handles). */
int64_t uaamg_total_launches(void);
/* Library-wide cap on device bytes held by all handles (0 = no cap), and the bytes held. */
int uaamg_set_memory_budget(uint64_t bytes);
uint64_t uaamg_memory_in_use(void);

const char* uaamg_status_string(int status);

/* ---- solve service ------------------------------------------------------------------- */
/*
 * A solve service on the current device (the serving extension of the method; the paper has
 * no counterpart).  Requests (CSR matrix, right-hand side, tolerance; host arrays, copied at
 * submit) are queued; `workers` host threads, each with its own CUDA stream, take them in
 * arrival order.  Hierarchies stay cached on the device, keyed by matrix_key (or, when it
 * is 0, a 64-bit FNV-1a hash of n and the three CSR arrays); least recently used idle ones
 * are freed to admit new ones within budget_bytes (0 = no budget), counted per service by
 * each hierarchy's admission estimate (the CSR, its coarse levels, setup scratch and the
 * solve workspace of up to max_batch columns).  While services with a budget live, the
 * library-wide cap of uaamg_set_memory_budget is the sum of their budgets.  A request whose
 * estimated hierarchy cannot fit the budget is answered with UAAMG_ERR_BUDGET; one that
 * fits after eviction waits until memory frees.  Continuous batching: a free worker takes,
 * in arrival order, every queued request whose matrix no other worker is using and whose
 * tolerance equals the oldest one's, up to max_batch <= 32 requests; requests for one matrix
 * become the columns of one system, and different matrices the systems of one
 * uaamg_solve_batch call (one system: uaamg_solve or uaamg_solve_many), so their K-cycles
 * advance level step by level step in shared launches.  Requests that arrive meanwhile wait
 * for the next free worker.  Each answer is the same algorithm as uaamg_solve on that
 * matrix (pre = post = 1; other sweep counts batch only requests of one matrix).
 */
typedef struct uaamg_server uaamg_server;
int uaamg_server_create(const uaamg_params* p, uint64_t budget_bytes, int32_t workers,
                        int32_t max_batch, uaamg_server** out);
/* A->on_device must be 0.  *ticket identifies the request for poll / wait. */
int uaamg_server_submit(uaamg_server* s, const uaamg_csr* A, uint64_t matrix_key,
                        const double* b, double tol, uint64_t* ticket);
int uaamg_server_poll(uaamg_server* s, uint64_t ticket, int32_t* done);
/* Blocks until the request is answered; x (host, n) receives the solution, latency_ms the
 * time from submit to answer, batch the number of requests solved together with it.
 * Returns the request's status; the ticket is released. */
int uaamg_server_wait(uaamg_server* s, uint64_t ticket, double* x, int32_t* iters,
                      double* relres, double* latency_ms, int32_t* batch);
/* Withdraws a request that no worker has taken yet: *cancelled = 1 and its wait returns
 * UAAMG_ERR_CANCELLED.  A request already being solved (or answered) is not interrupted:
 * *cancelled = 0 and its wait returns its result.  The ticket stays valid until waited on. */
int uaamg_server_cancel(uaamg_server* s, uint64_t ticket, int32_t* cancelled);
/* The answer of a request, with its time split: latency = queue (submit until a worker
 * took it) + setup (of its matrix, when the batch brought it; 0 for a cache hit) + solve
 * (the batch's solve) + hand-over. */
typedef struct uaamg_answer {
    int32_t status, iters, batch, cache_hit;
    double relres, latency_ms, queue_ms, setup_ms, solve_ms;
} uaamg_answer;
/* uaamg_server_wait that also fills *a (may be NULL); returns the request's status. */
int uaamg_server_wait_answer(uaamg_server* s, uint64_t ticket, double* x, uaamg_answer* a);
int uaamg_server_stats(uaamg_server* s, uint64_t* done, uint64_t* batches, uint64_t* cache_hits,
                       uint64_t* setups, uint64_t* rejected, int32_t* cached);
/* Finishes the queued requests, joins the workers and frees every cached hierarchy. */
void uaamg_server_destroy(uaamg_server* s);

/* ---- aggregation without device allocation ------------------------------------------ */
/*
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory (an external memory manager owns the device's memory, or the
 * calling thread must not issue cudaMalloc/cudaFree while other work is in flight).
 *
 * Aggregates one graph level exactly as level 0 of uaamg_setup does with agg_repeat = 1 and
 * sra_rounds = 0 (priorities, aggregation passes with size limit max_agg_size and pass_mode,
 * ascending coarse numbering; one aggregation stage, no subgraph reshaping) and writes
 * agg[i] = the coarse vertex of fine vertex i (device int32[n], caller-owned) and *nc (host)
 * = the number of aggregates.  A is validated like in uaamg_setup and must be on the device
 * (A->on_device = 1).  Nothing is allocated: all scratch lives in one static device array
 * of about 19 MB that every GPU loading this library holds until the process exits, so
 * A->n may be at most 262,144 (larger graphs return UAAMG_ERR_UNSUPPORTED before any device
 * work).  The first call on a device looks up that array's address (cudaGetSymbolAddress).
 * Every call shares the array and clears what must start at zero: calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and must be serialised by
 * the caller.  The call synchronises `stream` three times (after validation, after the
 * aggregation passes, and to read *nc).
 */
int uaamg_aggregate_static(const uaamg_csr* A, int32_t max_agg_size, int32_t pass_mode,
                           uint64_t seed, int32_t* agg, int32_t* nc, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* UAAMG_H */
