/*
 * CPU ORACLE -- test infrastructure, not part of the library.
 *
 * Plain, sequential FP64 C versions of what the CUDA library computes, written
 * straight from the definitions, so that a reader can check them against the
 * paper by eye.  The benchmark also builds this file with OpenMP, to time the
 * oracle on all host cores: then only the row loop of oracle_spmv is shared
 * among threads (static schedule); every row is still summed alone in
 * ascending order and everything else stays sequential, so both builds give
 * bitwise the same results.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use this file; the library never calls it, and it shares no code,
 * header or constant with the library's sources.
 *
 * Conventions: CSR as in the paper's Section 3.2 (CSR paragraph and the CSR
 * figure): `val` holds the nonzeros, `col_ind` their columns, `row_ptr[i]`
 * the offset of row i; the number of rows is len(row_ptr)-1 and the number of
 * columns is not stored.  All arithmetic is IEEE binary64, in the order the
 * definitions are written (ascending nonzero index, ascending vector index).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads an oracle_spmv call uses: 1 in the sequential build. */
int32_t oracle_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * spmv_csr (Section 3.2, CSR paragraph; the spmv_csr computation of
 * Section 2): for every row i, y[i] = sum over row_ptr[i] <= j < row_ptr[i+1]
 * of val[j] * x[col_ind[j]], accumulated in ascending j from 0.
 */
void oracle_spmv(int32_t rows, const int32_t* row_ptr, const int32_t* col_ind,
                 const double* val, const double* x, double* y) {
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < rows; ++i) {
        double s = 0.0;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) s += val[j] * x[col_ind[j]];
        y[i] = s;
    }
}

/*
 * dotproduct (Section 4.1, the dot-product computation in the robustness
 * figure): result = sum over 0 <= i < length of a[i] * b[i], ascending i.
 */
double oracle_dot(int64_t length, const double* a, const double* b) {
    double result = 0.0;
    for (int64_t i = 0; i < length; ++i) result += a[i] * b[i];
    return result;
}

/*
 * The "Maximum" invariant of Section 3.3 (data marshaling example): the
 * number of columns of a CSR matrix is max(col_ind) + 1 (0 if nnz == 0).
 */
int32_t oracle_csr_ncols(int64_t nnz, const int32_t* col_ind) {
    int32_t m = -1;
    for (int64_t j = 0; j < nnz; ++j)
        if (col_ind[j] > m) m = col_ind[j];
    return m + 1;
}

/* Status codes of oracle_cg. */
#define ORACLE_CG_CONVERGED 0
#define ORACLE_CG_MAXITER 1
#define ORACLE_CG_BREAKDOWN 2

/*
 * Unpreconditioned conjugate gradient (Hestenes & Stiefel, 1952), the solver
 * of the NAS CG benchmark whose SpMV loop the paper's compiler replaces
 * (Section 2, Figure 1; Section 5).  The paper does not print the solver;
 * this is the textbook iteration:
 *
 *   r = b - A x0;  p = r;  rr = r.r
 *   for k = 1 .. max_iter:
 *       q = A p;  pq = p.q
 *       if pq <= 0 or not finite: breakdown
 *       alpha = rr / pq
 *       x = x + alpha p;  r = r - alpha q
 *       rr_new = r.r
 *       if rr_new == 0 or sqrt(rr_new) <= rtol * ||b||: converged (k iterations)
 *       beta = rr_new / rr;  rr = rr_new
 *       p = r + beta p
 *
 * rtol <= 0 runs exactly max_iter iterations (stopping early only when
 * rr_new == 0).  x holds x0 on entry and the iterate on exit.  rr_hist
 * (nullable, max_iter+1 entries) receives rr before the first and after each
 * iteration.  Returns the status; *iters receives the iterations done.
 */
int oracle_cg(int32_t n, const int32_t* row_ptr, const int32_t* col_ind, const double* val,
              const double* b, double* x, int32_t max_iter, double rtol,
              int32_t* iters, double* rr_hist) {
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    int status = ORACLE_CG_MAXITER;
    int32_t k = 0;
    oracle_spmv(n, row_ptr, col_ind, val, x, q);
    for (int32_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rr = oracle_dot(n, r, r);
    double bnorm = sqrt(oracle_dot(n, b, b));
    if (rr_hist) rr_hist[0] = rr;
    if (rr == 0.0) status = ORACLE_CG_CONVERGED;
    while (status == ORACLE_CG_MAXITER && k < max_iter) {
        oracle_spmv(n, row_ptr, col_ind, val, p, q);
        double pq = oracle_dot(n, p, q);
        if (!(pq > 0.0) || !isfinite(pq)) { status = ORACLE_CG_BREAKDOWN; break; }
        double alpha = rr / pq;
        for (int32_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        double rr_new = oracle_dot(n, r, r);
        ++k;
        if (rr_hist) rr_hist[k] = rr_new;
        if (rr_new == 0.0 || (rtol > 0.0 && sqrt(rr_new) <= rtol * bnorm)) {
            status = ORACLE_CG_CONVERGED;
            break;
        }
        double beta = rr_new / rr;
        rr = rr_new;
        for (int32_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    *iters = k;
    free(r); free(p); free(q);
    return status;
}

/*
 * PageRank power iteration as in the GAP benchmark suite's PageRank kernel
 * that the paper accelerates (Section 5, Applications; Section 6.1, Graph
 * kernels: many SpMV calls on the same matrix).  The input is the TRANSPOSED
 * link matrix in CSR: row i lists the sources j of the edges j -> i with
 * value 1/outdeg(j).  A vertex whose column holds no entry has no out-edge
 * (it is dangling); its rank is spread uniformly over all N vertices.
 *
 *   x^0 = x0, or 1/N everywhere when x0 is NULL
 *   for t = 1 .. iters:
 *       D   = sum of x_j over dangling j
 *       y_i = d * (A^T x)_i + (d * D + 1 - d) / N
 *       l1[t-1] = sum_i |y_i - x_i|
 *       x = y
 *
 * The dangling set is found here from the matrix itself (empty columns).
 */
void oracle_pagerank(int32_t N, const int32_t* row_ptr, const int32_t* col_ind,
                     const double* val, const double* x0, int32_t iters, double d,
                     double* x_out, double* l1) {
    int64_t nnz = row_ptr[N];
    unsigned char* has_out = (unsigned char*)calloc((size_t)N, 1);
    double* x = (double*)malloc(sizeof(double) * (size_t)N);
    double* y = (double*)malloc(sizeof(double) * (size_t)N);
    for (int64_t j = 0; j < nnz; ++j) has_out[col_ind[j]] = 1;
    for (int32_t i = 0; i < N; ++i) x[i] = x0 ? x0[i] : 1.0 / (double)N;
    for (int32_t t = 0; t < iters; ++t) {
        double D = 0.0;
        for (int32_t j = 0; j < N; ++j)
            if (!has_out[j]) D += x[j];
        double teleport = (d * D + (1.0 - d)) / (double)N;
        oracle_spmv(N, row_ptr, col_ind, val, x, y);
        double s = 0.0;
        for (int32_t i = 0; i < N; ++i) {
            y[i] = d * y[i] + teleport;
            s += fabs(y[i] - x[i]);
        }
        if (l1) l1[t] = s;
        double* tmp = x; x = y; y = tmp;
    }
    memcpy(x_out, x, sizeof(double) * (size_t)N);
    free(has_out); free(x); free(y);
}

/*
 * Jagged Diagonal Storage (Section 3.2, JDS paragraph and the JDS figure):
 * rows are reordered by decreasing nonzero count; perm maps each original row
 * r to its slot perm[r] in that order (the reading under which the printed
 * example and the printed CSR example describe the same matrix); nzcnt[s] is
 * the count of slot s; the k-th nonzero of every slot that has one is stored
 * in jagged diagonal k, slots in order, and jd_ptr[k] is where diagonal k
 * starts.  Ties in the count keep the original row order (stable).  Within a
 * row the nonzeros keep their CSR order.  jd_ptr has max_row_length + 1
 * entries; returns the number of jagged diagonals.
 */
int32_t oracle_csr_to_jds(int32_t rows, const int32_t* row_ptr, const int32_t* col_ind,
                          const double* val, int32_t* perm, int32_t* nzcnt,
                          int32_t* jd_ptr, int32_t* jd_col, double* jd_val) {
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rows > 0 ? rows : 1));
    int32_t maxlen = 0;
    for (int32_t i = 0; i < rows; ++i) {
        order[i] = i;
        int32_t len = row_ptr[i + 1] - row_ptr[i];
        if (len > maxlen) maxlen = len;
    }
    /* stable insertion sort by decreasing length */
    for (int32_t i = 1; i < rows; ++i) {
        int32_t r = order[i];
        int32_t len = row_ptr[r + 1] - row_ptr[r];
        int32_t j = i - 1;
        while (j >= 0 && (row_ptr[order[j] + 1] - row_ptr[order[j]]) < len) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = r;
    }
    for (int32_t s = 0; s < rows; ++s) {
        perm[order[s]] = s;
        nzcnt[s] = row_ptr[order[s] + 1] - row_ptr[order[s]];
    }
    int32_t pos = 0;
    for (int32_t k = 0; k < maxlen; ++k) {
        jd_ptr[k] = pos;
        for (int32_t s = 0; s < rows && nzcnt[s] > k; ++s) {
            int32_t j = row_ptr[order[s]] + k;
            jd_col[pos] = col_ind[j];
            jd_val[pos] = val[j];
            ++pos;
        }
    }
    jd_ptr[maxlen] = pos;
    free(order);
    return maxlen;
}

/*
 * JDS SpMV (Section 3.2, the JDS computation of the JDS figure): for every
 * jagged diagonal k and every slot s < (length of diagonal k),
 * y[row of slot s] += val * x[col]; slots map back to rows through perm.
 * Accumulation per row in ascending k.
 */
void oracle_jds_spmv(int32_t rows, int32_t ndiag, const int32_t* perm, const int32_t* jd_ptr,
                     const int32_t* jd_col, const double* jd_val, const double* x, double* y) {
    int32_t* row_of_slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rows > 0 ? rows : 1));
    double* acc = (double*)calloc((size_t)(rows > 0 ? rows : 1), sizeof(double));
    for (int32_t r = 0; r < rows; ++r) row_of_slot[perm[r]] = r;
    for (int32_t k = 0; k < ndiag; ++k)
        for (int32_t s = 0; s < jd_ptr[k + 1] - jd_ptr[k]; ++s)
            acc[s] += jd_val[jd_ptr[k] + s] * x[jd_col[jd_ptr[k] + s]];
    for (int32_t s = 0; s < rows; ++s) y[row_of_slot[s]] = acc[s];
    free(row_of_slot);
    free(acc);
}

/*
 * Breadth-first search levels over a CSR adjacency (row i lists the
 * out-neighbours of i), the GAP BFS kernel of Section 5: level[src] = 0,
 * level[v] = 1 + min level of an in-neighbour, -1 if unreachable.  Plain
 * queue-based BFS.  Returns the number of reached vertices.
 */
int32_t oracle_bfs_levels(int32_t n, const int32_t* row_ptr, const int32_t* col_ind,
                          int32_t src, int32_t* level) {
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; ++i) level[i] = -1;
    int32_t head = 0, tail = 0;
    if (src >= 0 && src < n) { level[src] = 0; queue[tail++] = src; }
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int32_t v = col_ind[j];
            if (level[v] < 0) { level[v] = level[u] + 1; queue[tail++] = v; }
        }
    }
    free(queue);
    return tail;
}
