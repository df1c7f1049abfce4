// Batched kernels: many CSR problems of uneven size in one persistent launch.
//
// The work list holds (problem, tile) items for the SpMV phase and
// (problem, chunk) items for the vector phases of CG; persistent CTAs take
// items blockIdx.x, blockIdx.x + grid, ...  Every reduction of a problem is
// kept per item (one partial sum per tile or chunk) and added, in item order,
// by the CTA that completes the problem's last item (arrival counter), so a
// problem's result depends only on its own tiling -- the same alone and in
// any mix.  FP64 values and vectors.
#pragma once

#include "ops.cuh"

namespace lilac {

enum BatchKind : int { BK_SPMV = 0, BK_CG = 1 };

constexpr int kBatchThreads = 256;
constexpr int kBatchItems = 2048;   // nonzeros per tile: matches the STAGED tile list
constexpr int kBatchRows = 1024;    // rows per tile: matches the STAGED tile list
constexpr int kBatchChunk = 4096;   // vector elements per chunk item

struct BatchProb {
    // matrix (a handle's arrays and STAGED tile list)
    const int* row_ptr;
    const int* col_ind;
    const double* val;
    const TileDesc* tiles;
    const LongRow* longs;
    double* long_part;
    unsigned* long_cnt;
    double* long_red;
    int rows;
    int ntiles;
    int nlong;
    int kind;
    int nchunks;
    int pad;
    // SpMV: y = A x
    const double* x_in;
    double* y_out;
    // CG state and vectors
    const double* b;
    double* x;
    double* r;
    double* p;
    double* q;
    CgState* st;
    double rtol;
    int max_iter;
    int pad2;
    // per-item partial sums ([0, ntiles): SpMV phase; then nchunks) and the
    // arrival counters of the two reduction phases
    double* part;
    unsigned* cnt;
};

struct BatchItem {
    int prob;
    int idx;
};

// Item-order sum of a problem's partials (+ split-row sums), by one thread.
__device__ __forceinline__ double batch_sum_parts(const double* part, int n, const double* extra,
                                                  int nextra) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += __ldcg(part + i);
    for (int i = 0; i < nextra; ++i) s += __ldcg(extra + (size_t)i * kMaxRed);
    return s;
}

// SpMV phase: y = A x (BK_SPMV) or q = A p with p.q -> alpha (BK_CG).
static __global__ void __launch_bounds__(kBatchThreads)
    batch_spmv_kernel(const BatchProb* __restrict__ probs, const BatchItem* __restrict__ items,
                      const int* __restrict__ nitems_dev) {
    constexpr int THREADS = kBatchThreads;
    constexpr int IPT = kBatchItems / THREADS;
    constexpr int V = 4;
    constexpr int NGROUPS = THREADS / V;
    __shared__ double prod[kBatchItems];
    __shared__ int rp_s[kBatchRows + 2];
    __shared__ double sh[32];
    __shared__ double shr[kMaxRed * 32];
    const int tid = threadIdx.x;
    const int lane = tid & (V - 1), group = tid / V;
    const unsigned mask = group_mask<V>(tid);
    const int nitems = *nitems_dev;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const BatchProb& P = probs[item.prob];
        const int kind = P.kind;
        if (kind == BK_CG && cg_done(P.st)) continue;  // uniform over the block
        const TileDesc t = P.tiles[item.idx];
        const double* __restrict__ xin = kind == BK_CG ? P.p : P.x_in;
        double red = 0.0;
        // phase A: products of the tile's nonzeros
        int cj[IPT];
        double vj[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int k = t.k0 + j * THREADS + tid;
            cj[j] = k < t.k1 ? ld_stream(P.col_ind + k) : 0;
            vj[j] = k < t.k1 ? ld_stream(P.val + k) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int k = t.k0 + j * THREADS + tid;
            if (k < t.k1) prod[j * THREADS + tid] = vj[j] * __ldg(xin + cj[j]);
        }
        if (t.r1 >= 0) {
            const int nrows = t.r1 - t.r0;
            for (int q = tid; q <= nrows; q += THREADS) rp_s[q] = __ldg(P.row_ptr + t.r0 + q);
            __syncthreads();
            // phase B: rows of the tile
            for (int rr = group; rr < nrows; rr += NGROUPS) {
                const int kb = rp_s[rr] - t.k0, ke = rp_s[rr + 1] - t.k0;
                double sum = 0.0;
                for (int k = kb + lane; k < ke; k += V) sum += prod[k];
                sum = group_sum<V>(sum, mask);
                if (lane == 0) {
                    const int r = t.r0 + rr;
                    if (kind == BK_CG) {
                        P.q[r] = sum;
                        red += P.p[r] * sum;
                    } else {
                        P.y_out[r] = sum;
                    }
                }
            }
        } else {
            // chunk of a split row
            __syncthreads();
            double sum = 0.0;
            for (int k = tid; k < t.k1 - t.k0; k += THREADS) sum += prod[k];
            sum = block_sum_all<THREADS, double>(sum, sh);
            if (tid == 0) {
                const int lid = t.r0, slot = -t.r1 - 1;
                P.long_part[slot] = sum;
                __threadfence();
                const LongRow lr = P.longs[lid];
                if (atomicAdd(&P.long_cnt[lid], 1u) == (unsigned)lr.nchunks - 1u) {
                    __threadfence();
                    double rs = 0.0;
                    for (int j = 0; j < lr.nchunks; ++j) rs += __ldcg(&P.long_part[lr.first_slot + j]);
                    double lred = 0.0;
                    if (kind == BK_CG) {
                        P.q[lr.row] = rs;
                        lred = P.p[lr.row] * rs;
                    } else {
                        P.y_out[lr.row] = rs;
                    }
                    P.long_red[lid * kMaxRed] = lred;
                    P.long_cnt[lid] = 0u;
                }
            }
        }
        if (kind == BK_CG) {
            // this tile's share of p.q; the problem's last tile finishes alpha
            double r1[1] = {red}, tot[1];
            block_sum<1, THREADS>(r1, tot, shr);
            if (tid == 0) {
                P.part[item.idx] = tot[0];
                __threadfence();
                if (atomicAdd(&P.cnt[0], 1u) == (unsigned)P.ntiles - 1u) {
                    __threadfence();
                    const double pq = batch_sum_parts(P.part, P.ntiles, P.long_red, P.nlong);
                    P.st->pq = pq;
                    if (!(pq > 0.0) || !isfinite(pq)) {
                        P.st->status = LILAC_ERR_BREAKDOWN;
                        P.st->done = 1;
                    } else {
                        P.st->alpha = P.st->rr / pq;
                    }
                    P.cnt[0] = 0u;
                }
            }
        }
        __syncthreads();
    }
}

// Vector phases of CG over (problem, chunk) items.
//   PHASE 0: start   x = 0, r = p = b, rr = b.b
//   PHASE 1: update  x += alpha p, r -= alpha q, rr' = r.r -> beta, convergence
//   PHASE 2: direction p = r + beta p
template <int PHASE>
static __global__ void __launch_bounds__(kBatchThreads)
    batch_vec_kernel(const BatchProb* __restrict__ probs, const BatchItem* __restrict__ items,
                     const int* __restrict__ nitems_dev) {
    constexpr int THREADS = kBatchThreads;
    __shared__ double shr[kMaxRed * 32];
    const int tid = threadIdx.x;
    const int nitems = *nitems_dev;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const BatchProb& P = probs[item.prob];
        CgState* st = P.st;
        if (PHASE != 0 && cg_done(st)) continue;  // uniform over the block
        const int i0 = item.idx * kBatchChunk;
        const int i1 = min(P.rows, i0 + kBatchChunk);
        double red = 0.0;
        if (PHASE == 0) {
            for (int i = i0 + tid; i < i1; i += THREADS) {
                const double bi = P.b[i];
                P.x[i] = 0.0;
                P.r[i] = bi;
                P.p[i] = bi;
                red += bi * bi;
            }
        } else if (PHASE == 1) {
            const double alpha = st->alpha;
            for (int i = i0 + tid; i < i1; i += THREADS) {
                P.x[i] += alpha * P.p[i];
                const double ri = P.r[i] - alpha * P.q[i];
                P.r[i] = ri;
                red += ri * ri;
            }
        } else {
            const double beta = st->beta;
            for (int i = i0 + tid; i < i1; i += THREADS) P.p[i] = P.r[i] + beta * P.p[i];
            continue;  // no reduction
        }
        double r1[1] = {red}, tot[1];
        block_sum<1, THREADS>(r1, tot, shr);
        if (tid == 0) {
            P.part[P.ntiles + item.idx] = tot[0];
            __threadfence();
            if (atomicAdd(&P.cnt[1], 1u) == (unsigned)P.nchunks - 1u) {
                __threadfence();
                const double s = batch_sum_parts(P.part + P.ntiles, P.nchunks, nullptr, 0);
                if (PHASE == 0) {
                    st->rr = s;
                    st->bb = s;
                    st->tol2 = P.rtol > 0.0 ? P.rtol * P.rtol * s : -1.0;
                    st->iters = 0;
                    st->max_iter = P.max_iter;
                    st->done = s == 0.0 ? 1 : 0;
                    st->status = s == 0.0 ? LILAC_OK : LILAC_ERR_NOT_CONVERGED;
                } else {
                    const int iters = st->iters + 1;
                    st->iters = iters;
                    st->beta = s / st->rr;
                    st->rr = s;
                    if (s == 0.0 || (st->tol2 >= 0.0 && s <= st->tol2)) {
                        st->done = 1;
                        st->status = LILAC_OK;
                    } else if (iters >= st->max_iter) {
                        st->done = 1;
                        st->status = st->tol2 >= 0.0 ? LILAC_ERR_NOT_CONVERGED : LILAC_OK;
                    }
                }
                P.cnt[1] = 0u;
            }
        }
        __syncthreads();
    }
}

}  // namespace lilac
