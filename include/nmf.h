/*
 * nmf.h - C ABI of the GB300 multilevel nonnegative matrix factorisation library.
 *
 * Method: N. Gillis and F. Glineur, "A Multilevel Approach for Nonnegative
 * Matrix Factorization" (arXiv:1009.0881).  Given M >= 0 (m x n, one image of
 * an H x W pixel grid per column) and a rank r, the library computes V >= 0
 * (m x r) and W >= 0 (r x n) with M ~ VW (problem (NMF), Section 2), running
 * HALS (Algorithm HALS, Section 2.3), MU (Algorithm MU, Section 2.2) or ANLS
 * (Algorithm ANLS, Section 2.1 and Appendix A.2) sweeps inside the multigrid
 * cycles of Section 4.3 (V-cycle, nested iteration, full multigrid) over a
 * hierarchy of 2x2-coarsened pixel grids with the full-weighting restriction
 * of Eq. (4.1) and the prolongation of Eq. (4.2).
 *
 * Common conventions
 *  - All matrices are dense, row-major, float32, with no padding: M[i*n + j],
 *    V[i*r + k], W[k*n + j].  Pixel (y, x) of the grid is row y*grid_w + x.
 *  - A matrix pointer may address host memory (pageable or pinned) or device
 *    memory of the handle's device; the library asks the driver which
 *    (cudaPointerGetAttributes) and stages host data itself.  The caller owns
 *    every pointer it passes; the library never frees or keeps caller memory.
 *  - Every call runs on the handle's stream and has finished (results in
 *    place, host or device) when it returns.  A handle is not thread-safe:
 *    calls on one handle must not overlap.
 *  - Return values: NMF_OK (0) or a negative nmf_status; nmf_last_error()
 *    then returns a human-readable reason.  On error the output arrays are
 *    unspecified unless stated otherwise.
 *  - Limits: 1 <= r <= 64, m, n >= 1, 1 <= levels <= 16.
 */
#ifndef GB300_NMF_H
#define GB300_NMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmf_ctx* nmf_handle;

/* Inner NMF algorithm ("smoother") run at every level. */
typedef enum {
    NMF_HALS = 0, /* Algorithm HALS (Section 2.3): r exact column updates of V, then r row updates of W */
    NMF_MU = 1,   /* Algorithm MU (Section 2.2): Lee-Seung multiplicative updates */
    NMF_ANLS = 2, /* Algorithm ANLS (Section 2.1, Appendix A.2): exact NNLS for V then W (FP64 active set) */
    NMF_ANLS_BPP = 3 /* Algorithm ANLS with its NNLS problems solved by block principal pivoting (the
                        alternative the ANLS footnote of Section 2.1 names), FP64, started from the
                        support of the incoming row; rows where a passive block is numerically
                        singular, or where pivoting does not finish within 5r exchanges, are solved
                        by the active-set method instead */
} nmf_algo;

/* Storage precision of M and of the GEMM operands. */
typedef enum {
    NMF_FP32 = 0,     /* everything float32 */
    NMF_BF16 = 1,     /* M, V, W as bfloat16 GEMM operands, float32 accumulation and updates */
    NMF_BF16_FP32 = 2, /* NMF_BF16 for every sweep except the last quarter (at least one sweep) of the
                         last run of finest-level sweeps, which runs the float32 kernels on the
                         float32 M: the BF16 sweeps do most of the descent, the float32 ones remove
                         the bias that BF16 rounding of M leaves in the result.  With a stopping
                         rule (nmf_problem.rel_tol) only the float32 sweeps are watched. */
    NMF_AUTO = 3      /* per problem: NMF_BF16_FP32 for HALS and MU problems whose grid has at least
                         4096 pixels, NMF_FP32 otherwise (smaller grids, ANLS, and the entry points
                         that take no algorithm).  Measured on the uneven request pool of the
                         serving workload: below 64 x 64 pixels the float32 kernels (two launches
                         per sweep) finish a request sooner than the BF16 form (six launches per
                         sweep), and ANLS requests finish sooner in float32 at every size.  Under
                         a light load this lowers the latency; a saturated server completes fewer
                         requests per second than with NMF_BF16_FP32 (the float32 kernels take an
                         SM each and share the GPU less well between concurrent requests). */
} nmf_precision;

/* Multigrid cycle (Section 4.3). */
typedef enum {
    NMF_VCYCLE = 0, /* Algorithm V-cycle (Section 4.3.2) */
    NMF_NESTED = 1, /* Algorithm Nested Iteration (Section 4.3.1) */
    NMF_FMG = 2,    /* Algorithm Full Multigrid (Section 4.3.3) */
    NMF_WCYCLE = 3  /* W-cycle (a grid cycle Section 7 names as an extension): the V-cycle with the
                       coarser level visited twice in a row, each visit with sweep budget K/2 */
} nmf_cycle;

typedef enum {
    NMF_OK = 0,
    NMF_EINVAL = -1,   /* bad argument: sizes, m != grid_h*grid_w, r out of range, negative or NaN entries */
    NMF_ENOMEM = -2,   /* workspace would exceed the handle's HBM budget, or the device is out of memory */
    NMF_ENOCONV = -3,  /* an ANLS active-set solve hit its iteration cap (results are the last iterate) */
    NMF_ECUDA = -4,    /* a CUDA runtime call failed */
    NMF_ETIMEOUT = -5, /* a bounded device-side wait gave up */
    NMF_EBUSY = -6,    /* serving queue full or request not finished */
    NMF_ETOOBIG = -7   /* problem larger than the fixed scratch of nmf_error_noalloc */
} nmf_status;

/*
 * nmf_create - open a handle on CUDA device `device`.
 *   hbm_budget_bytes: upper bound on the device memory the handle may hold for
 *     its workspaces (0 = no limit besides the device's).  Work that needs more
 *     fails with NMF_ENOMEM before touching the device.
 *   prec: storage precision used by nmf_solve on this handle.
 *   *out receives the handle; release it with nmf_destroy.
 */
int nmf_create(nmf_handle* out, int device, size_t hbm_budget_bytes, nmf_precision prec);

/* nmf_destroy - free every device resource of the handle (NULL is accepted). */
void nmf_destroy(nmf_handle h);

/* nmf_last_error - reason for the last failing call on h (static string if h is NULL). */
const char* nmf_last_error(nmf_handle h);

/* Options of nmf_solve_ex.  Zero-initialise and set what is needed. */
typedef struct {
    nmf_cycle cycle;      /* multigrid cycle (default NMF_VCYCLE) */
    int64_t stop_after;   /* if > 0: run only the first stop_after sweeps of the schedule and
                             skip everything after them, transfers included (stopped in a run
                             on the finest level, the iterates are exactly those of the full run
                             at that point) */
    double* trace;        /* optional host array: ||M - VW||_F after each sweep at the finest level,
                             in schedule order; FP64 accumulation.  Costs one extra pass over M per
                             fine sweep. */
    int64_t trace_len;    /* capacity of trace; entries beyond it are not written */
    int64_t* trace_count; /* optional: receives the number of fine-level sweeps run */
    const int64_t* level_sweeps; /* optional: a V-cycle with these sweep counts per level instead of
                             the counts iters gives (Table 1): 2 levels - 1 entries in the order
                             the cycle runs them, before-sweeps of levels 1 .. L-1, the coarsest
                             level, after-sweeps of levels L-1 .. 1 (nmf_time_schedule computes
                             them from a time budget); each >= 0.  V-cycle only, not with
                             coarsen_columns (NMF_EINVAL). */
    int coarsen_columns;  /* nonzero: the columns of M form a sequence that varies smoothly
                             (Section 6.1: video frames, spectral bands) and are coarsened too:
                             level l has ceil(n_{l-1}/2) columns, M_{l+1} = R M_l R_n^T, and W
                             moves between levels along the sequence with the operators of
                             Eqs. (4.1) and (4.2) on an n x 1 grid, V over the pixel grid.
                             V-cycle and the FP32 form only (NMF_EINVAL otherwise). */
} nmf_options;

/*
 * nmf_solve - multilevel NMF (Section 4): improves (V, W) in place.
 *   M: m x n, M >= 0 (checked: NMF_EINVAL on a negative or NaN entry).
 *   grid_h * grid_w must equal m; rows are pixels in row-major grid order.
 *   r: factorisation rank, 1..64.
 *   algo: inner algorithm; levels: number of grid levels L (1 = the plain
 *   algorithm on the input grid); iters: sweep budget K.  With the reading of
 *   Table 1 (Section 4.3) a V-cycle runs floor(K/4) pre-sweeps and floor(K/2)
 *   post-sweeps on levels 1..L-1 and K sweeps on level L.
 *   V (m x r) and W (r x n): in = initial iterate (>= 0), out = result.
 * nmf_solve runs a V-cycle; nmf_solve_ex takes an nmf_options (NULL = defaults).
 */
int nmf_solve(nmf_handle h, const float* M, int64_t m, int64_t n, int grid_h, int grid_w,
              int r, nmf_algo algo, int levels, int iters, float* V, float* W);
int nmf_solve_ex(nmf_handle h, const float* M, int64_t m, int64_t n, int grid_h, int grid_w,
                 int r, nmf_algo algo, int levels, int iters, const nmf_options* opt,
                 float* V, float* W);

/* One problem of a batched solve (nmf_solve_batch). */
typedef struct {
    const float* M;    /* m x n, >= 0, host or device */
    int64_t m, n;
    int grid_h, grid_w; /* grid_h * grid_w == m */
    int r;
    nmf_algo algo;
    int levels, iters;  /* cycle levels L and sweep budget K, as in nmf_solve */
    nmf_cycle cycle;
    double rel_tol;     /* > 0: stopping rule on the last run of finest-level sweeps (the
                           post-smoothing of a V-cycle): stop once |f_{t-1} - f_t| <= rel_tol * f_t,
                           f_t = ||M - VW||_F after finest-level sweep t; 0: run the whole schedule */
    float* V;           /* in: V0 (m x r); out: result */
    float* W;           /* in: W0 (r x n); out: result */
    /* outputs */
    int status;         /* nmf_status of this problem */
    int64_t sweeps_run; /* sweeps executed over all levels */
    double objective;   /* ||M - VW||_F of the result, FP64 accumulation */
    /* input */
    const int64_t* level_sweeps; /* optional: explicit V-cycle counts as nmf_options.level_sweeps
                                    (2 levels - 1 entries, caller-owned until the call returns or
                                    the served request completes); NULL: the counts iters gives.
                                    Not taken by nmf_solve_grouped (NMF_EINVAL). */
} nmf_problem;

/*
 * nmf_solve_batch - solve `count` independent problems (any mix of sizes, ranks
 * and algorithms) at once: all of them are planned into one workspace and their
 * schedules recorded as concurrent branches of one CUDA graph, so the device
 * overlaps their kernels.  Each problem's result equals what nmf_solve would
 * return for it alone (same kernels, same launch shapes, same summation order),
 * up to the stopping rule.  Returns NMF_OK if every problem succeeded, else the
 * first failing status (per-problem statuses in probs[i].status).
 */
int nmf_solve_batch(nmf_handle h, nmf_problem* probs, int count);

/*
 * nmf_solve_grouped - the same problems as persistent grouped launches: every half-sweep of
 * the schedule (Section 4.3) is one launch whose CTAs (two per SM) take 64-row tiles of all
 * problems' factors from a work-list (the product with M over the whole of K, the HALS or
 * MU update of the tile's rows, the Gram slab of the new rows), after one launch that
 * reduces each problem's Gram slabs; the whole solve is one CUDA graph.  Problems that
 * meet their stopping rule do no further work (their tiles return as soon as they are taken).
 * Requirements (NMF_EINVAL otherwise): an NMF_FP32 or NMF_AUTO handle, algorithms NMF_HALS
 * or NMF_MU, and the same cycle, levels and iters for every problem; sizes and ranks may
 * differ.  A problem's result
 * does not depend on the rest of the group; it differs from nmf_solve's in the order of
 * the float32 sums (nmf_solve splits K across a thread-block cluster).  Outputs and
 * statuses as nmf_solve_batch.
 */
int nmf_solve_grouped(nmf_handle h, nmf_problem* probs, int count);

/*
 * nmf_workspace_bytes - device workspace nmf_solve_batch would hold on h for
 * the `count` problems probs[0..count-1] (no device work); negative nmf_status
 * on bad input.
 */
int64_t nmf_workspace_bytes(nmf_handle h, const nmf_problem* probs, int count);

/* nmf_release_workspace - free the handle's device workspace (and its cached graphs). */
int nmf_release_workspace(nmf_handle h);

/*
 * Serving form: a request loop with continuous batching.  `slots` worker slots
 * each own a handle (stream + workspace).  Submitted requests wait in a FIFO
 * queue; a free slot takes the longest run of requests from the head (at most
 * 16) whose combined workspace fits in the HBM budget (sum of the workspaces
 * held by all slots <= hbm_budget_bytes; idle slots release theirs when the
 * queue head does not fit) and solves them as one nmf_solve_batch, on its own
 * stream while other slots run theirs.  A request's result is the one
 * nmf_solve_batch gives it alone.  The environment variable NMF_SERVE_MAX_BATCH
 * (1..16, read at nmf_server_create) lowers the number of requests a slot takes at
 * once: a batch is one CUDA graph per combination of request shapes, so 1 reuses
 * the graph of each shape and leaves the overlap to the slots' streams.
 */
typedef struct nmf_server_s* nmf_server;
int nmf_server_create(nmf_server* out, int device, size_t hbm_budget_bytes, int slots, nmf_precision prec);
/* Queue *prob (which must stay valid until its ticket completes); returns a ticket >= 0,
   or NMF_ENOMEM if the problem alone exceeds the budget, NMF_EINVAL on bad input. */
int64_t nmf_server_submit(nmf_server s, nmf_problem* prob);
/* NMF_OK once the ticket completed (outputs in its nmf_problem; *latency_ms, if not NULL,
   receives submit-to-completion time), NMF_EBUSY if not within wait_ms (-1 = wait forever). */
int nmf_server_poll(nmf_server s, int64_t ticket, int wait_ms, double* latency_ms);
/* Counters: queued, running, completed requests and device bytes held by the slots. */
int nmf_server_stats(nmf_server s, int64_t* queued, int64_t* running, int64_t* completed, int64_t* bytes_held);
/* Waits for queued and running requests, then frees everything. */
void nmf_server_destroy(nmf_server s);

/*
 * nmf_error - ||M - VW||_F (problem (NMF), Section 2) with float32 products;
 * each thread sums four squared residuals of a row in float32 and the
 * accumulation of those sums is FP64.  *err_out receives the value (host
 * pointer).
 */
int nmf_error(nmf_handle h, const float* M, const float* V, const float* W,
              int64_t m, int64_t n, int r, double* err_out);

/*
 * nmf_schedule - host-side sweep allocation of a cycle (no device work).
 *   Writes the number of sweeps run on each level 1..levels into
 *   sweeps_per_level[0..levels-1] (Table 1 of Section 4.3 for the V-cycle and
 *   nested iteration; Algorithm FMG's recursion for NMF_FMG; for NMF_WCYCLE two
 *   coarser visits of budget K/2 in place of the V-cycle's one) and returns the
 *   total, or a negative nmf_status.
 */
int64_t nmf_schedule(nmf_cycle cycle, int levels, int iters, int64_t* sweeps_per_level);

/*
 * nmf_time_schedule - host-side split of a V-cycle's time budget over its levels (no device
 * work).  Algorithm V-cycle (Section 4.3) gives a level with time T_l a quarter of it for
 * sweeps before the restriction, a quarter for the coarser cycle and half for sweeps after
 * the prolongation; the coarsest level spends all of its T_L.  With T_1 = budget and the
 * cost of one sweep on level l in costs[l-1] (same unit as budget, > 0), level l < L runs
 * floor(T_l / (4 costs[l-1])) sweeps before and floor(T_l / (2 costs[l-1])) after, the
 * coarsest floor(T_L / costs[L-1]).  Table 1 is this split when every level's sweep costs a
 * quarter of the one above (then the counts are floor(K/4), K, floor(K/2) for
 * budget = K costs[0]).  Writes the 2 levels - 1 counts in the order the cycle runs them
 * (before-sweeps of levels 1 .. L-1, the coarsest level, after-sweeps of levels L-1 .. 1)
 * to level_sweeps_out, for nmf_options.level_sweeps.  Returns NMF_OK or NMF_EINVAL.
 */
int nmf_time_schedule(int levels, double budget, const double* costs, int64_t* level_sweeps_out);

/*
 * nmf_restrict - Y = R X, the full-weighting restriction of Eq. (4.1) applied
 * to each of the `cols` columns of X ((grid_h*grid_w) x cols).  Y is
 * (ceil(grid_h/2)*ceil(grid_w/2)) x cols.  On the border the stencil keeps the
 * in-bounds fine pixels and renormalises their weights to sum 1.
 */
int nmf_restrict(nmf_handle h, const float* X, int grid_h, int grid_w, int64_t cols, float* Y);

/*
 * nmf_prolong - X = P Y, the prolongation of Eq. (4.2) from the coarse grid
 * (ceil(grid_h/2) x ceil(grid_w/2)) to the fine grid grid_h x grid_w, for each
 * of the `cols` columns.  A fine pixel is the mean of its 1, 2 or 4 coarse
 * neighbours (neighbours past an even-size border are dropped).
 */
int nmf_prolong(nmf_handle h, const float* Y, int grid_h, int grid_w, int64_t cols, float* X);

/*
 * nmf_products - the four dense products of one HALS/MU sweep (Section 2.3,
 * Appendix A.1) with the library's GEMM kernels:
 *   A = M W^T (m x r), B = W W^T (r x r), C = V^T M (r x n), D = V^T V (r x r).
 * Any output pointer may be NULL to skip it.
 */
int nmf_products(nmf_handle h, const float* M, const float* V, const float* W,
                 int64_t m, int64_t n, int r, float* A, float* B, float* C, float* D);

/*
 * nmf_sweep - `sweeps` iterations of the inner algorithm at a single level
 * (no grid): identical to nmf_solve with levels = 1, grid m x 1.
 */
int nmf_sweep(nmf_handle h, const float* M, int64_t m, int64_t n, int r, nmf_algo algo,
              int sweeps, float* V, float* W);

/* nmf_device_info - number of SMs of the handle's device and the library's build tag. */
int nmf_device_info(nmf_handle h, int* num_sms, const char** build_tag);

/*
 * nmf_set_stream - run the handle's work on `stream` (a cudaStream_t of the
 * handle's device, passed as void*; NULL restores the handle's own stream).
 * The caller keeps ownership of the stream.  Calls stay synchronous.
 */
int nmf_set_stream(nmf_handle h, void* stream);

/*
 * nmf_set_limits - bounds of the iterative and waiting parts of a solve on h.
 *   nnls_max_exchanges: cap on the variables an ANLS active-set solve may add
 *     to its passive set per row (Appendix A.2; the reading used here caps the
 *     outer loop at 3r).  A row that reaches the cap keeps its last iterate
 *     (feasible, >= 0) and the call returns NMF_ENOCONV.  < 0: the default 3r.
 *   barrier_spins: polls of a grid-wide barrier in the persistent kernels
 *     before it gives up; the kernel then leaves, the call returns NMF_ETIMEOUT
 *     and the handle stays usable.  < 0: the default (about a second).
 * Takes effect for later calls on h (cached CUDA graphs are dropped).  Small
 * values exist to exercise those two failure paths.
 */
int nmf_set_limits(nmf_handle h, int nnls_max_exchanges, int64_t barrier_spins);

/*
 * nmf_last_launch_count - number of kernels the last successful call on h
 * launched (graph kernel nodes included), or a negative nmf_status.
 */
int64_t nmf_last_launch_count(nmf_handle h);

/*
 * nmf_profile_sweep - per-kernel timing of one sweep at a single level:
 * each phase is launched `reps` times on the handle's stream between CUDA
 * events, and ms_out[i] receives the mean duration of one launch, in order:
 *   [0] products for the V-step (A = M W^T and B = W W^T, one launch)
 *   [1] V-step update        [2] products for the W-step (C = V^T M, D = V^T V)
 *   [3] W-step update        [4] error evaluation ||M - VW||_F
 * M, V, W as in nmf_sweep; they are read only (the library works on copies).
 */
int nmf_profile_sweep(nmf_handle h, const float* M, int64_t m, int64_t n, int r, nmf_algo algo,
                      const float* V, const float* W, int reps, float* ms_out);

/*
 * nmf_profile_coarse - timing of the persistent coarse-level kernel, which a
 * solve uses for the HALS / MU sweeps (Algorithms 2 and 3) on coarse levels
 * (Section 4.2) of the FP32 form whose V has at most 32 rows: one untimed run,
 * then one run of `sweeps` sweeps between CUDA events on the handle's stream;
 * *ms_out receives the mean time of one sweep.  M (m x n), V, W as in
 * nmf_sweep, read only.  NMF_EINVAL if the kernel does not apply to this
 * shape, algorithm or precision (or NMF_COARSE=0 disables it).
 */
int nmf_profile_coarse(nmf_handle h, const float* M, int64_t m, int64_t n, int r, nmf_algo algo,
                       const float* V, const float* W, int sweeps, float* ms_out);

/*
 * nmf_error_noalloc - ||M - VW||_F, the same value as nmf_error, computed
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as a
 * service that reserved all of the GPU's memory up front for its own pool, or
 * a latency-bound loop that cannot afford the implicit device synchronisation
 * of cudaMalloc/cudaFree.  It needs no handle and calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 *   M (m x n), V (m x r), W (r x n): device (or managed) pointers on the
 *     calling thread's current device, dense row-major float32 (the caller's
 *     layout, no copy); a host pointer or another device's memory gives
 *     NMF_EINVAL.
 *   stream: cudaStream_t (as void*) to run on; NULL = the default stream.
 *   err_out: host pointer; receives the norm.  The call returns once it is written.
 *
 * Scratch: the per-tile partial sums live in one fixed device array of
 * 65537 doubles (512 KiB + 8 bytes), a file-scope __device__ variable of the
 * library; every GPU that loads the library holds it until the process
 * exits.  Its capacity is 65536 tiles of 64 x 64 entries of M, i.e.
 * ceil(m/64) * ceil(n/64) <= 65536 (for example m = n = 16384); larger
 * problems are rejected with NMF_ETOOBIG before any work is queued.
 * Every call looks the array's device address up (cudaGetSymbolAddress, on
 * the calling thread's current device); nothing is cached between calls, so a
 * device reset leaves no stale address behind.  The first call on a device
 * may load the library's device code there: make it before any CUDA stream
 * capture begins.
 * All calls on a device share the array and each call overwrites what it
 * uses, so calls whose GPU work overlaps (different streams or threads at
 * the same time) race and can return wrong values: serialise them.
 * Returns NMF_OK, NMF_EINVAL (null or non-device pointer, m or n < 1, r
 * outside 1..64), NMF_ETOOBIG, or NMF_ECUDA.
 */
int nmf_error_noalloc(const float* M, const float* V, const float* W, int64_t m, int64_t n, int r,
                      void* stream, double* err_out);

#ifdef __cplusplus
}
#endif

#endif /* GB300_NMF_H */
