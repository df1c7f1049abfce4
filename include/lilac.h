/*
 * lilac.h -- C ABI of the GB300 sparse library: CSR sparse matrix-vector
 * multiply on a device-resident matrix, and the two loops built on it that
 * the paper accelerates, conjugate gradient and PageRank.
 *
 * Paper: P. Ginsbach, B. Collie, M. F. P. O'Boyle, "Automatically Harnessing
 * Sparse Acceleration", CC 2020 (arXiv 2001.07938).
 *
 *  - The arguments of the SpMV entry points are those of the paper's
 *    spmv_csr computation (Section 3.2, CSR paragraph: rows, row_ptr,
 *    col_ind, val, x -> y); the paper's LiLAC-What program names them as
 *    the harness interface (Section 3.1).
 *  - The paper's persistent harness state and data marshaling (Section 3.3:
 *    PersistentVariables / BeforeFirstExecution / AfterLastExecution,
 *    Marshaling with CudaRead; Section 4.2: the construct / update /
 *    destruct contract of ReadObject) become an explicit handle:
 *    lilac_csr_create uploads the matrix once (construct + update),
 *    lilac_csr_update_values re-uploads changed values (update), and
 *    lilac_csr_destroy frees it (destruct).  The library keeps no pointer
 *    to caller memory; it copies what it needs.
 *  - The data-dependent invariant the paper caches (the column count
 *    "cols" = Maximum(col_ind), Section 3.3) is computed once at create,
 *    together with the row-length statistics and the tile schedule the
 *    kernels use, and the dangling-vertex set PageRank needs (on first use).
 *
 * Conventions for every entry point:
 *  - Every function returns a lilac_status; no exception crosses the ABI
 *    (a failed host allocation returns LILAC_ERR_OOM, any other internal
 *    failure LILAC_ERR_CUDA).  lilac_last_error() gives a one-line message
 *    for the calling thread's last failure.
 *  - Indices are int32 and 0-based; nnz < 2^31.  Empty rows are allowed
 *    (their y is 0), so are duplicate (i, j) entries (they add up) and
 *    unsorted columns.
 *  - `stream` is a cudaStream_t (NULL: the legacy default stream).  Device
 *    vectors are caller-owned and must not alias each other.  Work is
 *    stream-ordered and asynchronous unless a call says it synchronizes.
 *  - A handle may be used from one stream at a time: two calls on the same
 *    handle must not run concurrently on different streams (they share the
 *    handle's scratch memory).
 *  - A call that fails on the device (a bounded wait that timed out) marks
 *    the handle; later calls return LILAC_ERR_TIMEOUT until
 *    lilac_csr_reset_error().
 */
#ifndef LILAC_H
#define LILAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lilac_csr_s* lilac_csr; /* opaque; owned by the library */

typedef enum {
    LILAC_OK = 0,
    LILAC_ERR_INVALID_ARG = 1,   /* NULL handle/pointer, negative size, bad option */
    LILAC_ERR_INVALID_CSR = 2,   /* row_ptr not monotone / not 0..nnz, col_ind out of range */
    LILAC_ERR_OOM = 3,           /* device allocation failed */
    LILAC_ERR_BUDGET = 4,        /* request exceeds a configured device-memory budget */
    LILAC_ERR_CUDA = 5,          /* a CUDA runtime call failed (see lilac_last_error) */
    LILAC_ERR_BREAKDOWN = 6,     /* CG: p.Ap <= 0 or not finite (matrix not SPD) */
    LILAC_ERR_NOT_CONVERGED = 7, /* CG: tolerance not reached within max_iter */
    LILAC_ERR_TIMEOUT = 8,       /* a device-side bounded wait gave up */
    LILAC_ERR_DTYPE = 9,         /* operation not defined for the handle's value type */
    LILAC_ERR_UNSUPPORTED = 10   /* feature not available in this build or device */
} lilac_status;

typedef enum { LILAC_F64 = 0, LILAC_F32 = 1 } lilac_dtype;
typedef enum { LILAC_MEM_HOST = 0, LILAC_MEM_DEVICE = 1 } lilac_mem;

/* SpMV kernel variants (all compute the same y; they differ in how rows and
 * nonzeros map to threads). */
typedef enum {
    LILAC_VARIANT_AUTO = 0,   /* chosen at create from row-length statistics */
    LILAC_VARIANT_SCALAR = 1, /* one thread per row */
    LILAC_VARIANT_VECTOR = 2, /* V lanes per row, V in {2,4,8,16,32}; V = 32 is warp-per-row */
    LILAC_VARIANT_STAGED = 3, /* nnz-balanced row tiles staged in shared memory by bulk
                                 asynchronous copies; rows longer than a tile are split */
    LILAC_VARIANT_MERGE = 4,  /* merge-path partition of (rows + nonzeros) over CTAs; each thread
                                 walks 8 consecutive path items, rows split between threads or
                                 CTAs are finished from carries; no lanes-per-row setting */
    LILAC_VARIANT_SLAB = 5,   /* column slabs, built once per matrix: one CTA per SM holds a
                                 slab of x (up to 192 KB) in shared memory and runs the sliced
                                 ELL chunks of that slab's pieces of one group of rows (each
                                 row's piece summed by one lane); the last of a group's CTAs
                                 adds the pieces in slab order and runs the epilogue.  Inside
                                 FP64 CG the CTAs take equal runs of their slab's pieces and
                                 leave q as the slab partials, which the CG update adds.
                                 Matrices with more than 64 slabs, or whose pieces pad by more
                                 than a quarter, run STAGED */
    LILAC_VARIANT_JDS = 6,    /* jagged diagonal storage (Section 3.2), built once per matrix:
                                 rows sorted by length, one thread per row, nonzero d of all
                                 rows stored together; on another value array (an FP32 copy)
                                 STAGED runs */
    LILAC_VARIANT_SELL = 7,   /* sliced ELL (chunks of 32 rows, element k of the chunk's 32
                                 rows stored together), built once per matrix: one lane per row
                                 with one fused multiply-add per nonzero; rows longer than a
                                 piece cap are cut into pieces finished in piece order; rows
                                 sorted by length when row order would pad much.  On another
                                 value array (an FP32 copy), or where the copy would pad by more
                                 than half, STAGED runs */
    LILAC_VARIANT_HUB = 8     /* hub columns, built once per matrix, for power-law matrices whose x
                                 exceeds 1 MB: the most frequent columns (up to 4 slabs of 192 KB
                                 of x, while a slab adds 5% of the nonzeros) are gathered once
                                 per call and held in shared memory, one CTA per SM summing each
                                 row's piece of its slab; the other nonzeros run as a sliced ELL
                                 copy whose lanes add the slab sums before the epilogue.  Where
                                 the hub columns hold under 40% of the nonzeros, or on another
                                 value array, STAGED runs */
} lilac_variant;

/* lilac_csr_create flags.  By default create times the candidate SpMV
 * variants once on the matrix and keeps the fastest (the one-off tuning
 * phase of an autotuning sparse library, paid at create like the paper's
 * cached invariants). */
#define LILAC_CREATE_NO_TUNE 0x1u /* skip the timing; keep the choice made from row statistics */
/* The choice from row statistics (mean row length m, coefficient of variation
 * cv, longest row): short regular rows (m <= 12, cv <= 1): STAGED with one
 * lane per row; irregular rows (cv > 1, or a row longer than a 2048-nonzero
 * tile) and other short rows: STAGED with min(w, 8) lanes per row, w the
 * smallest power of two >= m / 2; long regular rows: VECTOR with the smallest
 * power of two >= m / 16 lanes per row (2 .. 32).  The timed trial starts
 * from this choice and keeps it unless another candidate is faster; a
 * sliced ELL candidate (SELL, SLAB, HUB) within 3% of the fastest counts as
 * a tie and is kept (its solver forms are the cheaper ones). */

/*
 * Upload a CSR matrix once and return a handle (construct + update of the
 * paper's marshaling contract, Section 4.2).
 *   rows     number of rows, >= 0 (the length of row_ptr minus one, Section 3.2)
 *   ncols    number of columns; < 0 means max(col_ind) + 1 (the Maximum
 *            invariant of Section 3.3; 0 when nnz == 0)
 *   nnz      number of stored entries, 0 <= nnz < 2^31; must equal row_ptr[rows]
 *   row_ptr  rows + 1 int32 offsets, row_ptr[0] == 0, non-decreasing
 *   col_ind  nnz int32 column indices in [0, ncols)
 *   vals     nnz values of type `dtype` (double for LILAC_F64, float for LILAC_F32)
 *   where    whether the three arrays are in host or device memory
 *   flags    LILAC_CREATE_* bits
 *   stream   stream for the upload; the call synchronizes it before returning
 *   out      receives the handle (NULL on failure)
 * The arrays are copied; the caller may free or change them afterwards.
 * Errors: INVALID_ARG, INVALID_CSR (validated on the device), OOM, CUDA.
 */
lilac_status lilac_csr_create(int32_t rows, int32_t ncols, int64_t nnz, const int32_t* row_ptr,
                              const int32_t* col_ind, const void* vals, lilac_dtype dtype,
                              lilac_mem where, uint32_t flags, void* stream, lilac_csr* out);

/*
 * Replace the values (same structure): the paper's "update" step, run when
 * the data of a marshaled array changed (Section 4.2).  nnz values of the
 * handle's dtype.  Asynchronous on `stream`.  Cached FP32 copies derived
 * from FP64 values are refreshed.
 */
lilac_status lilac_csr_update_values(lilac_csr A, const void* vals, lilac_mem where, void* stream);

/* Free everything the handle owns (the paper's "destruct").  NULL is a no-op.
 * Synchronizes the device work the handle issued. */
lilac_status lilac_csr_destroy(lilac_csr A);

typedef struct {
    int32_t rows;
    int32_t ncols;
    int64_t nnz;
    int32_t dtype;          /* lilac_dtype */
    int32_t variant;        /* lilac_variant in use */
    int32_t vector_width;   /* lanes per row for VECTOR / STAGED; for SLAB / SELL, the
                               STAGED width used on another value array */
    int32_t max_row_len;
    int32_t empty_rows;
    int32_t num_tiles;      /* STAGED: row tiles incl. long-row chunks */
    int32_t num_long_rows;  /* STAGED: rows split across tiles */
    int32_t sm_count;
    double mean_row_len;
    double std_row_len;
    int64_t device_bytes;   /* device memory held by the handle right now */
    int64_t h2d_bytes;      /* bytes uploaded to the matrix so far (create + updates) */
    int32_t active_variant; /* the kernel that runs on the handle's own values: `variant`, or
                               STAGED where a SLAB / SELL / JDS copy does not suit the matrix */
    int32_t sell_split_rows; /* SELL copy: rows cut into pieces (0 without a copy) */
    int64_t sell_padded_nnz; /* SELL copy: stored elements including padding (0 without one) */
    int32_t spmv_kernels;    /* kernels one SpMV with a reducing epilogue (CG, PageRank) launches
                                on the handle's own values: 2 for SELL on many sorted short rows
                                (SpMV + row-order reduction), else 1 */
} lilac_csr_info_t;

/* Describe the handle.  Synchronous only on host state. */
lilac_status lilac_csr_info(lilac_csr A, lilac_csr_info_t* info);

/* Override the autotuner: variant (lilac_variant, not AUTO) and, for VECTOR
 * and STAGED, lanes per row (power of two 1..32; 0 keeps the current one;
 * SCALAR, MERGE and JDS use 1 whatever is passed; for SLAB and SELL it is the
 * STAGED width used where they fall back to STAGED).  Affects later calls.
 * Choosing SLAB, SELL or JDS builds that copy of the matrix on first use
 * (synchronous; errors OOM, CUDA); a matrix the copy does not suit runs
 * STAGED. */
lilac_status lilac_csr_set_variant(lilac_csr A, int32_t variant, int32_t vector_width);

/* The autotuner's trial on this handle (the tuning phase that an autotuning
 * library runs once per matrix, Section 5 (SparseX); the paper's finding that
 * no single implementation wins, Section 6.2): candidate i ran variant
 * `variants[i]` at `widths[i]` lanes per row in `ms[i]` milliseconds per call
 * (y = A x, the fastest of two rounds of three calls, after two warm-up
 * calls), in the order tried.  Up to `max` entries are written to the
 * caller's host arrays (NULL skips an array); *n receives the number of
 * candidates, 0 when the handle was created with LILAC_CREATE_NO_TUNE or is
 * empty.  Host state only: no synchronisation.  Errors: INVALID_ARG (NULL
 * handle or n, max < 0). */
lilac_status lilac_csr_tune_table(lilac_csr A, int32_t max, int32_t* variants, int32_t* widths,
                                  float* ms, int32_t* n);

/*
 * The handle's jagged diagonal storage (the JDS format of Section 3.2), built
 * on first use of LILAC_VARIANT_JDS or by this call (synchronous), copied to
 * host buffers (NULL pointers are skipped):
 *   perm     rows entries: perm[r] = slot of row r; rows are sorted by length,
 *            longest first, rows of equal length in row order
 *   jd_ptr   max_row_len + 1 entries: jagged diagonal d holds the d-th nonzero
 *            of every row longer than d, at [jd_ptr[d], jd_ptr[d+1]), by slot
 *   col_ind, vals  nnz entries (vals in the handle's dtype), JDS order
 *   nzcnt    rows entries: nonzeros of the row in slot s
 * Errors: INVALID_ARG, OOM, CUDA.
 */
lilac_status lilac_csr_jds(lilac_csr A, int32_t* perm, int32_t* jd_ptr, int32_t* col_ind,
                           void* vals, int32_t* nzcnt);

/*
 * y = A x (the paper's spmv_csr computation, Section 3.2):
 *   y[i] = sum over row_ptr[i] <= j < row_ptr[i+1] of val[j] * x[col_ind[j]].
 *   x  ncols elements, y  rows elements, both of the handle's dtype; FP64
 *      matrices accumulate in FP64, FP32 matrices in FP32.
 *   where  LILAC_MEM_DEVICE: x and y are device pointers; the call is
 *          asynchronous.  LILAC_MEM_HOST: x and y are host pointers; the
 *          library copies x in and y out through its own device buffers and
 *          synchronizes `stream` before returning (pinned host memory makes
 *          the copies asynchronous DMA).
 * Errors: INVALID_ARG, CUDA, TIMEOUT.
 */
lilac_status lilac_spmv(lilac_csr A, const void* x, void* y, lilac_mem where, void* stream);

typedef struct {
    int32_t max_iter;       /* iteration cap (precisions 0 and 2) or outer-refinement cap (1) */
    double rtol;            /* stop when ||r|| <= rtol ||b||; <= 0: run exactly max_iter */
    int32_t precision;      /* 0: FP64 CG.  1: FP32 inner CG + FP64 iterative refinement.
                               2: FP32 CG with FP64 reliable updates (x += d and the
                               residual replaced by b - A x, both in FP64, whenever the
                               FP32 residual fell by ru_delta; the search direction is kept) */
    double inner_rtol;      /* mixed: inner stop ||r_in|| <= inner_rtol ||r_outer|| */
    int32_t inner_max_iter; /* mixed: inner iteration cap per refinement */
    int32_t use_x0;         /* 1: start from x as given; 0: start from x = 0 */
    int32_t true_residual;  /* 1: recompute ||b - A x|| / ||b|| in FP64 at the end */
    int32_t use_graph;      /* 1: replay the iterations as a captured CUDA graph */
    int32_t check_every;    /* iterations between host convergence checks when rtol > 0 */
    int32_t profile;        /* 1: time every SpMV launch of the solve with CUDA events
                               (reported in lilac_cg_info; needs info) */
    double ru_delta;        /* precision 2: replacement threshold in (0, 1) */
} lilac_cg_opts;

typedef struct {
    int32_t iters;          /* CG iterations done (all inner iterations when mixed) */
    int32_t refinements;    /* precision 1: outer refinement steps; 2: residual replacements */
    int32_t status;         /* lilac_status of the solve */
    int32_t pad;
    double rel_res;         /* recursive (FP64 CG) or outer true (mixed) ||r|| / ||b|| */
    double true_rel_res;    /* ||b - A x|| / ||b|| in FP64 if requested, else -1 */
    double spmv_ms;         /* opts->profile: summed duration of the SpMV launches */
    int32_t spmv_launches;  /* opts->profile: number of SpMV launches timed */
    int32_t kernel_launches; /* kernels the solve launched (including no-op ones after convergence) */
} lilac_cg_info;

/* Fill *o with the defaults: max_iter 1000, rtol 1e-10, FP64, inner_rtol
 * 1e-5, inner_max_iter 1000, use_x0 0, true_residual 1, use_graph 1,
 * check_every 32, profile 0, ru_delta 0.1. */
void lilac_cg_opts_default(lilac_cg_opts* o);

/*
 * Solve A x = b for symmetric positive definite A with unpreconditioned
 * conjugate gradient (Hestenes-Stiefel; the NAS CG solver whose SpMV loop
 * the paper's compiler replaces, Section 2 and Section 5).  Each iteration is
 * q = A p with p.q fused into the SpMV; x += alpha p, r -= alpha q with r.r
 * fused into one pass; p = r + beta p.  The scalars stay on the device.
 *   b, x    rows FP64 elements; x holds x0 on entry if opts->use_x0, the
 *           solution on exit.  `where` as in lilac_spmv.
 *   opts    NULL: defaults.  Precisions 1 and 2 run the FP32 iterations on
 *           FP32 values (the handle's, or an FP32 copy derived once from
 *           FP64 values) and compute the FP64 residual b - A x with the
 *           handle's own values; their rel_res is that FP64 residual.
 *   info    nullable; if given, the call synchronizes `stream` at the end.
 * Returns OK, NOT_CONVERGED (rtol > 0 not reached), BREAKDOWN, or an error.
 * With rtol > 0 the call synchronizes `stream` every check_every iterations.
 */
lilac_status lilac_cg(lilac_csr A, const double* b, double* x, lilac_mem where,
                      const lilac_cg_opts* opts, lilac_cg_info* info, void* stream);

/*
 * PageRank power iteration (the GAP PageRank kernel the paper accelerates,
 * Section 5 and Section 6.1) on the TRANSPOSED link matrix: row i lists the
 * sources j of the edges j -> i with value 1/outdeg(j); a vertex whose
 * column is empty has no out-edge (dangling) and its rank is spread
 * uniformly.  Per iteration, with N = rows and D = sum of x_j over dangling j:
 *     y_i = d * (A x)_i + (d * D + 1 - d) / N,    l1_t = sum_i |y_i - x_i|,   x = y.
 *   x             N elements of the handle's dtype: the start vector on entry
 *                 (unless init_uniform, which starts from 1/N), the result on exit
 *   iters         number of iterations (>= 0), no early stop
 *   damping       d in [0, 1]
 *   l1_per_iter   nullable host array of iters doubles; if given, the call
 *                 synchronizes `stream` and copies the per-iteration L1 changes
 * Row sums, y and x are in the handle's dtype; D and L1 are accumulated in
 * FP64.  Needs rows == ncols.
 */
lilac_status lilac_pagerank(lilac_csr AT, void* x, int32_t init_uniform, int32_t iters,
                            double damping, double* l1_per_iter, lilac_mem where, void* stream);

/*
 * Y = A X for k right-hand sides at once (multi-vector SpMV, 1 <= k <= 32):
 * every nonzero is streamed once for all k vectors (no counterpart in the
 * paper, whose spmv_csr takes one vector; it serves batches of SpMV requests).
 *   X  ncols x k, Y  rows x k, both of the handle's dtype, host or device per
 *      `where`.  layout LILAC_LAYOUT_ROWS: element (i, j) at [i * k + j] (the
 *      k values of one row adjacent, the kernel's own layout);
 *      LILAC_LAYOUT_VECTORS: at [j * n + i] (k separate vectors, as lilac_spmv
 *      takes them; transposed through device scratch).
 * Each row's sums use their own summation order (tolerance as lilac_spmv).
 * Asynchronous for device pointers.  Errors: INVALID_ARG, OOM, CUDA.
 */
typedef enum { LILAC_LAYOUT_ROWS = 0, LILAC_LAYOUT_VECTORS = 1 } lilac_layout;
lilac_status lilac_spmm(lilac_csr A, const void* X, void* Y, int32_t k, int32_t layout,
                        lilac_mem where, void* stream);

/*
 * The paper's harness calling convention: y = A x on the caller's own host
 * arrays with no handle (spmv_csr, Section 3.1), the marshaling done by the
 * library (Sections 3.3 and 4.2).
 *   mode LILAC_HOST_CACHED: the library keeps a resident copy per distinct
 *        (row_ptr, col_ind, vals, rows, ncols, nnz, dtype) and decides what
 *        changed since it was uploaded: `version` != 0 is the caller's version
 *        number of the three arrays (the number of the previous call =
 *        unchanged, nothing is read); otherwise (version 0, or a new number)
 *        the library hashes the arrays' contents (a host pass over them) and
 *        compares with the hashes of the upload.  Changed structure rebuilds
 *        the copy; changed values alone are re-uploaded.
 *        At most 32 copies are kept (least recently used evicted).
 *   mode LILAC_HOST_NAIVE: create (kernel chosen from row statistics, no
 *        timed tuning), upload, multiply and free on every call (the naive
 *        insertion the paper measures against, Section 6.3).
 *   ncols < 0: max(col_ind) + 1.  x (ncols) and y (rows) are host arrays of
 *   `dtype`; the call synchronizes `stream`.  The paper's page-protection
 *   change tracking is not reproduced: writes the caller hides behind an
 *   unchanged version number are not seen.
 * Thread-safe (one lock around the cache).  Errors as lilac_csr_create and
 * lilac_spmv.
 */
typedef enum { LILAC_HOST_CACHED = 0, LILAC_HOST_NAIVE = 1 } lilac_host_mode;

typedef struct {
    int64_t calls;             /* lilac_spmv_host calls */
    int64_t uploads;           /* resident copies created (every call when naive) */
    int64_t value_updates;     /* calls that re-uploaded values only */
    int64_t structure_changes; /* calls that found a changed structure */
    int64_t hits;              /* calls that reused a copy unchanged */
    int64_t hashed_bytes;      /* host bytes hashed by version-0 calls */
    int32_t resident;          /* copies held now */
    int32_t pad;
} lilac_host_stats_t;

lilac_status lilac_spmv_host(int32_t rows, int32_t ncols, int64_t nnz, const int32_t* row_ptr,
                             const int32_t* col_ind, const void* vals, lilac_dtype dtype,
                             const void* x, void* y, uint64_t version, uint32_t mode, void* stream);
/* Counters of the host-convention cache since the last clear. */
lilac_status lilac_host_cache_stats(lilac_host_stats_t* st);
/* Free every resident copy of the host-convention cache and zero its counters. */
lilac_status lilac_host_cache_clear(void);

/*
 * Breadth-first search levels from `source` on the TRANSPOSED adjacency
 * matrix (row v lists the sources u of the edges u -> v, as for
 * lilac_pagerank; values are ignored): the GAP BFS kernel of Section 5, run
 * as one masked boolean SpMV per level (an unvisited v joins level L+1 when
 * one of its in-neighbours is at level L).
 *   level   rows int32 (host or device per `where`): level of every vertex,
 *           0 for the source, -1 if unreachable.  The levels are unique, so
 *           any correct BFS gives the same array.
 *   depth   nullable: number of levels (1 + the largest level).
 * Needs rows == ncols.  Synchronizes `stream` every 8 levels.  Errors:
 * INVALID_ARG (source not a vertex, level NULL), OOM, CUDA.
 */
lilac_status lilac_bfs(lilac_csr AT, int32_t source, int32_t* level, lilac_mem where,
                       int32_t* depth, void* stream);

/*
 * y = A x on CSR arrays the caller already holds on the device, with no
 * device allocation.  The paper has no counterpart: this is for callers that
 * must not call cudaMalloc -- e.g. code running while another component owns
 * the device memory through its own pool and budget, or a latency-critical
 * loop where cudaMalloc / cudaFree (which can synchronise the device) are
 * not acceptable -- and that therefore cannot create a handle.
 *   rows, ncols, nnz   sizes; rows + nnz < 2^31 (else LILAC_ERR_INVALID_ARG)
 *   row_ptr, col_ind, vals, x, y   device pointers, caller-owned; the arrays
 *                      must form valid CSR (row_ptr[0] = 0, non-decreasing,
 *                      row_ptr[rows] = nnz, 0 <= col_ind < ncols): nothing is
 *                      validated, and invalid arrays are read out of range
 *   dtype              type of vals, x and y (FP64 accumulates in FP64, FP32 in FP32)
 *   stream             cudaStream_t; the call is asynchronous
 * Runs the MERGE kernel with its scratch (carry records, per-CTA partial sums,
 * arrival counter; 82,176 bytes, room for the at most 2048 CTA ranges a call
 * launches whatever the size) in one fixed array in device memory that every
 * GPU loading this library holds until the process exits.  The only size
 * refused is rows + nnz >= 2^31.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current, and
 * where modules load lazily it also loads the library's kernels and their
 * array onto the device, which allocates and can synchronise: make that first
 * call a warm-up outside the latency-critical loop and before any stream
 * capture.  The address is kept for the life of the process, so resetting
 * the device (cudaDeviceReset) after the first call is not supported.  Every
 * call shares the array: calls whose kernels overlap on the GPU (e.g. on two
 * streams at once) race and give wrong results.  Each call clears the counter
 * that must start at zero.
 */
lilac_status lilac_spmv_noalloc(int32_t rows, int32_t ncols, int64_t nnz, const int32_t* row_ptr,
                                const int32_t* col_ind, const void* vals, lilac_dtype dtype,
                                const void* x, void* y, void* stream);

/*
 * Kernel timing switch.  enable != 0 starts timing every SpMV launch that
 * later lilac_cg / lilac_pagerank calls on this handle make (CUDA event pairs
 * recorded on the launching stream, also inside captured graphs; the calls
 * then synchronise their stream) and clears the totals.  enable == 0 stops
 * and returns, in *spmv_ms and *spmv_launches (both nullable), the summed
 * duration and number of the SpMV launches timed since it was enabled.
 */
lilac_status lilac_csr_profile(lilac_csr A, int32_t enable, double* spmv_ms, int64_t* spmv_launches);

/*
 * Batched execution: many problems of uneven size (FP64 or FP32 handles) in
 * one persistent launch per phase (beyond the paper, which issues one library
 * call per detected loop; batching many small problems addresses the paper's
 * finding that small sizes are not profitable alone, Section 6.2).  The work
 * list holds one kind of item per problem, following the kernel the handle's
 * autotuner chose (the paper's finding that no single implementation wins,
 * Section 6.2): groups of eight chunks of the sliced ELL copy for handles
 * tuned to SELL or SLAB (the copy is built on first batched use; SLAB's
 * column slabs need a whole SM each, so its problems run the sliced ELL form
 * of the same layout), the STAGED tiles for the others and where the copy
 * does not hold the values multiplied (an FP64 handle's FP32 values).
 * Every reduction of a problem is kept per item and added in
 * item order, so a problem's result is bitwise the same alone and in any
 * batch.
 */
typedef struct lilac_batch_s* lilac_batch;

/* Create a batch context on the current device (work lists, workspace arena,
 * captured rounds).  Not thread-safe; one context per host thread. */
lilac_status lilac_batch_create(lilac_batch* out);
lilac_status lilac_batch_destroy(lilac_batch B); /* NULL is a no-op */

/* y[i] = A[i] x[i] for i < count: device vectors of A[i]'s value type
 * (double for FP64 handles, float for FP32 ones; y[i] of A[i]'s rows, x[i]
 * of its columns); A[i] may repeat.  Asynchronous on `stream` after a short
 * synchronous set-up of the work lists (and, on first use of a handle, of
 * its sliced ELL copy). */
lilac_status lilac_batch_spmv(lilac_batch B, int32_t count, const lilac_csr* A,
                              const void* const* x, void* const* y, void* stream);

/* CG on count systems A[i] x[i] = b[i] at once (x0 = 0), each stopping at
 * ||r|| <= rtol ||b|| (rtol <= 0: exactly max_iter iterations); iterations
 * of all systems run together in captured rounds of 16, with one host check
 * per round.  precision 0: FP64; 2: FP32 values and vectors with FP64
 * reliable updates (as lilac_cg precision 2, residual replaced when it fell
 * by 0.1; FP32 values derived once per handle).  infos (nullable) receives
 * per-system iterations, status, residual replacements and relative residual
 * (recursive for FP64, the last FP64 b - A x for precision 2).  FP32 handles
 * take precision 2 only (their own values are the FP32 values; the FP64
 * residual promotes them), else LILAC_ERR_DTYPE.  b and x are FP64 device
 * vectors for every handle.  Returns OK or the first non-OK status. */
lilac_status lilac_batch_cg(lilac_batch B, int32_t count, const lilac_csr* A,
                            const double* const* b, double* const* x, int32_t max_iter,
                            double rtol, int32_t precision, lilac_cg_info* infos, void* stream);

/*
 * Request server: continuous batching of SpMV and FP64 CG requests over a
 * pool of matrices kept resident on the device under a memory budget -- the
 * paper's marshaling (upload once, keep resident, free when needed; Section
 * 3.3, Section 4.2) applied to a stream of requests.  Single-threaded: the
 * caller submits requests as they arrive and calls lilac_server_step in its
 * loop.  Each step admits queued requests in arrival order while the budget
 * and the active limit allow (uploading a matrix on first use and evicting
 * the least recently used idle matrix when memory is needed, for the matrix
 * or for a request's workspace), runs one round and retires finished
 * requests (result copied to the caller's host buffer).  A round has two
 * lanes.  Requests on matrices of fewer than 2^19 nonzeros run batched:
 * every single-vector SpMV in one launch, iters_per_round iterations of every
 * CG solve in one captured graph.  On a second stream, concurrently, SpMV
 * requests of 2 to 32 vectors run through the multi-vector kernel (each
 * nonzero streamed once for all its vectors), and single-vector SpMVs and CG
 * solves on larger matrices run the matrix's own tuned kernels (lilac_spmv's
 * and lilac_cg's, iters_per_round iterations per round).  The lane depends
 * on the request alone, so a request's result is bitwise the same whatever
 * else is in flight.  A request that cannot fit the budget even with nothing
 * else in flight completes with LILAC_ERR_BUDGET.
 */
typedef struct lilac_server_s* lilac_server;

typedef struct {
    int64_t hbm_budget_bytes; /* resident matrices + request workspaces (default 120 GiB) */
    int32_t max_active;       /* requests in flight at most (default 256) */
    int32_t iters_per_round;  /* CG iterations per step (default 16) */
    int32_t tune;             /* 1: time the SpMV variants of a matrix at its first upload (the
                                 autotuner of lilac_csr_create); 0 (default): row statistics */
} lilac_server_opts;

typedef enum { LILAC_REQ_SPMV = 0, LILAC_REQ_CG = 1 } lilac_req_kind;

typedef struct {
    int32_t kind;      /* lilac_req_kind */
    int32_t matrix;    /* id from lilac_server_add_matrix */
    int32_t nvec;      /* SpMV: number of vectors (>= 1) */
    int32_t max_iter;  /* CG: iteration cap (>= 1) */
    double rtol;       /* CG: stop at ||r|| <= rtol ||b|| (<= 0: run max_iter) */
    const double* in;  /* host: SpMV x, nvec x ncols (vector-major); CG b, rows */
    double* out;       /* host: SpMV y, nvec x rows; CG x, rows; written before completion */
    int64_t tag;       /* caller's id, returned in the completion */
    int32_t precision; /* CG: 0 FP64; 2 FP32 values and vectors with FP64 reliable
                          updates (as lilac_cg precision 2; FP32 values derived once) */
    int32_t pad;
} lilac_request;

typedef struct {
    int64_t tag;
    int32_t status;    /* lilac_status of the request */
    int32_t iters;     /* CG iterations */
    double rel_res;    /* CG recursive ||r|| / ||b|| */
    double arrival;    /* lilac_server_now() at submit */
    double finish;     /* lilac_server_now() at retirement */
    double admitted;   /* lilac_server_now() when it left the queue (workspace granted) */
    int32_t rounds;    /* server steps it took part in */
    int32_t pad;
} lilac_completion;

typedef struct {
    int64_t submitted, completed, rounds, uploads, upload_bytes, evictions, budget_waits;
    int64_t resident_bytes, pool_bytes;
    int32_t queued, active;
} lilac_server_stats_t;

void lilac_server_opts_default(lilac_server_opts* o);
/* Create on the current device; `stream` carries the server's uploads and
 * batched work (the large-matrix lane runs on a stream the server creates and
 * orders after it).  Errors: INVALID_ARG (options), CUDA (stream creation). */
lilac_status lilac_server_create(const lilac_server_opts* o, void* stream, lilac_server* out);
/* Free everything (in-flight requests are dropped).  NULL is a no-op. */
lilac_status lilac_server_destroy(lilac_server S);
/* Register an FP64 CSR matrix by its host arrays, which must stay valid and
 * unchanged until the server is destroyed (they are uploaded on demand). */
lilac_status lilac_server_add_matrix(lilac_server S, int32_t rows, int32_t ncols, int64_t nnz,
                                     const int32_t* row_ptr, const int32_t* col_ind,
                                     const double* vals, int32_t* id);
/* Queue a request (host only; `in` and `out` must stay valid until its
 * completion is polled).  Errors: INVALID_ARG, BUDGET (matrix alone exceeds it). */
lilac_status lilac_server_submit(lilac_server S, const lilac_request* r);
/* One round (admission, batched launches, retirement); synchronizes the
 * server's stream.  *pending (nullable) = requests queued or active after it. */
lilac_status lilac_server_step(lilac_server S, int32_t* pending);
/* Take up to max completions (oldest first); *n receives how many. */
lilac_status lilac_server_poll(lilac_server S, lilac_completion* out, int32_t max, int32_t* n);
lilac_status lilac_server_stats(lilac_server S, lilac_server_stats_t* st);
/* The server's clock (seconds, monotonic). */
double lilac_server_now(void);

/* Clear a sticky device error of the handle and re-zero its scratch memory. */
lilac_status lilac_csr_reset_error(lilac_csr A);

/*
 * Test hooks for the failure paths (no counterpart in the paper; for tests of
 * error handling, which must not fault a shared GPU):
 *   LILAC_INJECT_ALLOC_FAIL, arg n >= 1: the n-th device allocation from now
 *       (process-wide; A may be NULL) fails with LILAC_ERR_OOM; arg 0 cancels.
 *   LILAC_INJECT_SKIP_COPY (arg unused): the next STAGED SpMV launch of A
 *       leaves the first bulk copy of its first CTA unissued, so that CTA's
 *       bounded wait expires after about 2 s; the CTA records a device
 *       timeout and returns, and A reports LILAC_ERR_TIMEOUT from its next
 *       synchronizing call until lilac_csr_reset_error.  Every wait in the
 *       kernels is bounded, so nothing hangs or faults.
 *   LILAC_INJECT_SKIP_BARRIER (arg unused): in the next fused CG step of A
 *       (FP64 CG on a SLAB handle), CTA 0 does not arrive at the step's grid
 *       barrier; the other CTAs give up after about 2 s and record a device
 *       timeout, reported as above.
 */
typedef enum {
    LILAC_INJECT_ALLOC_FAIL = 1,
    LILAC_INJECT_SKIP_COPY = 2,
    LILAC_INJECT_SKIP_BARRIER = 3
} lilac_inject;
lilac_status lilac_debug_inject(lilac_csr A, int32_t what, int64_t arg);

/* Static text for a status code. */
const char* lilac_status_string(lilac_status s);

/* Message of the calling thread's last failed call ("" if none). */
const char* lilac_last_error(void);

/* ABI version of this header: major * 10000 + minor * 100 + patch. */
int32_t lilac_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LILAC_H */
