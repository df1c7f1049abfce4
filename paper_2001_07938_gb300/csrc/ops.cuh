// Epilogues fused into the SpMV kernels, and the vector kernels of the CG
// and PageRank loops.  Device scalars live in small state structs so that a
// whole solve runs without the host reading anything between iterations.
#pragma once

#include <cmath>

#include "../../include/lilac.h"
#include "spmv_kernels.cuh"

namespace lilac {

// ---------------------------------------------------------------------------
// Plain y = A x.
template <class V, class T>
struct OpStore {
    using ValT = V;
    using VecT = T;
    using AccT = T;
    using RedT = double;
    static constexpr int NR = 0;
    static constexpr bool kTwoPhase = true;
    T* __restrict__ y;
    __device__ bool skip() const { return false; }
    __device__ void begin() {}
    __device__ void row(int r, AccT s, RedT*) const { y[r] = s; }
    __device__ void store(int r, AccT s) const { y[r] = s; }
    __device__ void reduce(int, RedT*) const {}
    __device__ void finish(const double*) const {}
};

// ---------------------------------------------------------------------------
// Conjugate gradient (Hestenes-Stiefel).  State of one solve on the device.
struct CgState {
    double rr;       // r.r of the current residual
    double pq;       // p.Ap of the last iteration
    double alpha;
    double beta;
    double bb;       // b.b (right-hand side of this solve)
    double tol2;     // stop when rr <= tol2 (negative: never)
    double true_rr;  // ||b - A x||^2 recomputed at the end (if asked)
    double scale;    // mixed precision: 1 / ||r_outer|| used to scale the inner rhs
    int iters;       // iterations completed
    int max_iter;
    int done;        // 1: later iteration kernels are no-ops
    int status;      // lilac_status of the solve so far
    // mixed precision with reliable updates
    double rr_anchor;  // FP32 residual r.r right after the last replacement
    double delta2;     // replace when r.r <= delta2 * rr_anchor
    int update;        // 1: this iteration replaces r by the FP64 residual
    int updates;       // replacements done
    int dir_iter;      // -1: no direction waits for a replaced residual (kept for the layout)
    int pad_;
};

__device__ __forceinline__ bool cg_done(const CgState* st) {
    return *reinterpret_cast<const volatile int*>(&st->done) != 0;
}

// q = A p with p.q fused: after the grid sum, alpha = rr / p.q.
template <class V, class T>
struct OpCgPq {
    using ValT = V;
    using VecT = T;
    using AccT = T;
    using RedT = typename RedOf<T>::type;
    static constexpr int NR = 1;
    static constexpr bool kTwoPhase = true;
    T* __restrict__ q;
    const T* __restrict__ p;
    CgState* st;
    __device__ bool skip() const { return cg_done(st); }
    __device__ void begin() {}
    __device__ void row(int r, AccT s, RedT* red) const {
        q[r] = s;
        red_add_prod(red[0], p[r], s);
    }
    __device__ void store(int r, AccT s) const { q[r] = s; }
    __device__ void reduce(int r, RedT* red) const { red_add_prod(red[0], p[r], __ldcg(q + r)); }
    __device__ void finish(const double* tot) const {
        const double pq = tot[0];
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->status = LILAC_ERR_BREAKDOWN;
            st->done = 1;
        } else {
            st->alpha = st->rr / pq;
        }
    }
};

// Residual r = b - A x in FP64 (values of any type promoted), with r.r and
// b.b.  Mode INIT starts a CG solve from x0 (also p = r); mode TRUE only
// records ||b - A x||^2; mode OUTER starts a refinement step (r kept in
// FP64, scale = 1/||r||, convergence test against rtol ||b||).
enum ResidualMode { RES_INIT = 0, RES_TRUE = 1, RES_OUTER = 2 };

template <class V, int MODE>
struct OpResidual {
    using ValT = V;
    using VecT = double;
    using AccT = double;
    using RedT = double;
    static constexpr int NR = 2;
    static constexpr bool kTwoPhase = false;
    double* __restrict__ r;
    double* __restrict__ p;  // INIT only
    const double* __restrict__ b;
    CgState* st;
    double rtol;
    __device__ bool skip() const { return false; }
    __device__ void begin() {}
    __device__ void row(int i, AccT s, double* red) const {
        const double bi = b[i];
        const double ri = bi - s;
        if (MODE != RES_TRUE) r[i] = ri;
        if (MODE == RES_INIT) p[i] = ri;
        red[0] += ri * ri;
        red[1] += bi * bi;
    }
    __device__ void finish(const double* tot) const {
        if (MODE == RES_TRUE) {
            st->true_rr = tot[0];
            st->bb = tot[1];
            return;
        }
        st->rr = tot[0];
        st->bb = tot[1];
        st->tol2 = rtol > 0.0 ? rtol * rtol * tot[1] : -1.0;
        st->iters = 0;
        if (MODE == RES_OUTER) {
            st->scale = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
            const bool conv = tot[0] == 0.0 || tot[0] <= st->tol2;
            st->done = conv ? 1 : 0;
            st->status = conv ? LILAC_OK : LILAC_ERR_NOT_CONVERGED;
        } else {
            const bool conv = tot[0] == 0.0 || (st->tol2 >= 0.0 && tot[0] <= st->tol2);
            st->done = conv ? 1 : 0;
            st->status = conv ? LILAC_OK : LILAC_ERR_NOT_CONVERGED;
        }
    }
};

// ---------------------------------------------------------------------------
// Vector kernels of CG.  Persistent grid-stride loops; grid sums through the
// ticket.  THREADS is fixed at 256.
constexpr int kVecThreads = 256;

struct FinNone {
    __device__ void finish(const double*) const {}
};

// x = 0, r = b, p = b (cast to T), rr = b.b: start of a solve from x0 = 0.
template <class T>
struct FinCgStart {
    CgState* st;
    double rtol;
    __device__ void finish(const double* tot) const {
        st->rr = tot[0];
        st->bb = tot[0];
        st->tol2 = rtol > 0.0 ? rtol * rtol * tot[0] : -1.0;
        st->iters = 0;
        const bool conv = tot[0] == 0.0;
        st->done = conv ? 1 : 0;
        st->status = conv ? LILAC_OK : LILAC_ERR_NOT_CONVERGED;
    }
};

template <class T, class TB>
static __global__ void __launch_bounds__(kVecThreads)
    cg_start_zero_kernel(int n, const TB* __restrict__ b, double bscale, T* __restrict__ x,
                         T* __restrict__ r, T* __restrict__ p, FinCgStart<T> fin, Scratch s) {
    double red[1] = {0.0};
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads) {
        const T bi = T(double(b[i]) * bscale);
        x[i] = T(0);
        r[i] = bi;
        p[i] = bi;
        red[0] += double(bi) * double(bi);
    }
    grid_reduce_finish<1, kVecThreads>(fin, red, s, 0);
}

// 16-byte vector of T: the CG vector kernels move four FP32 or two FP64
// elements per access when every array is 16-byte aligned.
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int N = 4;
    __device__ static float get(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
    __device__ static void set(float4& v, int i, float a) {
        if (i == 0) v.x = a; else if (i == 1) v.y = a; else if (i == 2) v.z = a; else v.w = a;
    }
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int N = 2;
    __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
    __device__ static void set(double2& v, int i, double a) {
        if (i == 0) v.x = a; else v.y = a;
    }
};

__device__ __forceinline__ bool aligned16(const void* a, const void* b, const void* c = nullptr,
                                          const void* d = nullptr) {
    return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
             reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
}

// SLAB, CG form: one FP64 CG step q = A p with p.q, leaving the ends of the
// step to cg_step_slabs_kernel, which follows.  q is left as the S slab partials
// P[s][row]: the update adds them in slab order where it reads q (the same
// sums as the row-group combine of spmv_slab_kernel).  p.q is taken from the
// pieces instead of the rows: lane l of chunk c keeps t = p[row] * piece (0
// on padding lanes), and each CTA adds the t of its own chunks in chunk
// order, so no CTA waits for the other slabs of its rows.  That frees the
// CTAs from row groups: `ranges` gives each CTA a run of its slab's chunks
// with about equal padded element counts, and warps take the run's chunks
// from a shared counter.  The t live in shared memory after the slab when
// they fit (tsm), else in T.  The CTA's sum goes to slot blockIdx.x of
// s.partials and the kernel ends there, with no grid ticket:
// cg_step_slabs_kernel adds the slots (fixed order) and takes alpha.
template <int THREADS, int UNR>
__global__ void __launch_bounds__(THREADS, 1)
    spmv_slab_cg_kernel(SlabView V, const int4* __restrict__ ranges, int tsm,
                        const double* __restrict__ sval, const double* __restrict__ p,
                        double* __restrict__ P, double* __restrict__ T, const CgState* st,
                        Scratch s) {
    if (cg_done(st)) return;
    extern __shared__ __align__(16) unsigned char slab_smem[];
    __shared__ int next_chunk;
    double* xs = reinterpret_cast<double*>(slab_smem);
    const int4 c = ranges[blockIdx.x];  // {slab, first chunk, end chunk, -}
    const int sl = c.x;
    const int c0 = sl * V.W;
    slab_load_x<THREADS>(xs, p, c0, min(V.W, V.ncols - c0), V.W);
    // the chunk lanes' p[row] * piece: after the slab (and its zero) in
    // shared memory, 16-byte aligned, or in T
    double* ts = tsm ? xs + ((V.W + 2) & ~1) : T + (size_t)c.y * 32;
    if (threadIdx.x == 0) next_chunk = c.y + THREADS / 32;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double* __restrict__ Ps = P + (size_t)sl * V.rows;
    int ch = c.y + (int)(threadIdx.x >> 5);
    while (ch < c.z) {
        const int row = __ldg(V.crow + (size_t)ch * 32 + lane);
        const double acc = slab_chunk_sum<UNR, kSlabPipe, double>(V, sval, xs, ch, lane);
        double t = 0.0;
        if (row >= 0) {
            Ps[row] = acc;
            t = __ldg(p + row) * acc;
        }
        ts[(ch - c.y) * 32 + lane] = t;
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&next_chunk, 1);
        ch = __shfl_sync(0xffffffffu, nx, 0);
    }
    __syncthreads();  // this CTA's t are written and visible to the block
    double red[1] = {0.0};
    const int nt = (c.z - c.y) * 32;
    for (int i = (int)threadIdx.x; i < nt; i += THREADS) red[0] += tsm ? ts[i] : __ldcg(ts + i);
    // block sum with the second level in warp 0 only: FP64 adds take the
    // narrow FP64 pipe, so no thread repeats the warps' sum
    __shared__ double sh[32];
    double tot[1];
    block_sum<1, THREADS>(red, tot, sh);
    if (threadIdx.x == 0) s.partials[blockIdx.x] = tot[0];
}


// ---------------------------------------------------------------------------
// Mixed precision with reliable updates (residual replacement, in the manner
// of van der Vorst & Ye, "Residual replacement strategies for Krylov subspace
// iterative methods for the convergence of true residuals", SISC 2000): one
// FP32 CG whose correction d accumulates in FP32; when its recursive residual
// has fallen by delta since the last replacement (or reaches the tolerance,
// or the iteration cap), x += d in FP64, d = 0, and r is replaced by
// float(b - A x) computed in FP64, keeping the search direction (the CG step
// took beta from the recursive r and formed p before the replacement).

// A replacement flagged by the CG step, in a solve that is not finished.
__device__ __forceinline__ bool ru_due(const CgState* st) {
    return *reinterpret_cast<const volatile int*>(&st->update) != 0 && !cg_done(st);
}

// r = float(b - A x) with b - A x in FP64 (values of any type promoted);
// ||b - A x||^2 decides convergence, float(r).float(r) is the new r.r (beta
// is recorded too but no longer read: the direction was formed already).
template <class V>
struct OpResidualRU {
    using ValT = V;
    using VecT = double;
    using AccT = double;
    using RedT = double;
    static constexpr int NR = 2;
    static constexpr bool kTwoPhase = false;
    float* __restrict__ r;
    const double* __restrict__ b;
    CgState* st;
    __device__ bool skip() const { return !ru_due(st); }
    __device__ void begin() {}
    __device__ void row(int i, AccT s, double* red) const {
        const double ri = b[i] - s;
        const float rf = float(ri);
        r[i] = rf;
        red[0] += ri * ri;
        red[1] += double(rf) * double(rf);
    }
    __device__ void finish(const double* tot) const {
        st->true_rr = tot[0];
        st->updates += 1;
        st->update = 0;
        if (tot[0] == 0.0 || (st->tol2 >= 0.0 && tot[0] <= st->tol2)) {
            st->done = 1;
            st->status = LILAC_OK;
        } else if (st->iters >= st->max_iter) {
            st->done = 1;
            st->status = st->tol2 >= 0.0 ? LILAC_ERR_NOT_CONVERGED : LILAC_OK;
        } else {
            st->beta = tot[1] / st->rr;  // r.r before this iteration
            st->rr = tot[1];
            st->rr_anchor = tot[1];
        }
    }
};

// Start: r = p = float(r64), d = 0, r.r (after an FP64 residual r64 = b - A x0).
struct FinRuStart {
    CgState* st;
    double delta2;
    __device__ void finish(const double* tot) const {
        st->rr = tot[0];
        st->rr_anchor = tot[0];
        st->delta2 = delta2;
        st->update = 0;
        st->updates = 0;
        st->iters = 0;
        st->true_rr = st->bb > 0.0 ? -1.0 : 0.0;
    }
};

static __global__ void __launch_bounds__(kVecThreads)
    ru_start_kernel(int n, const double* __restrict__ r64, float* __restrict__ r,
                    float* __restrict__ p, float* __restrict__ d, FinRuStart fin, Scratch s) {
    double red[1] = {0.0};
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads) {
        const float rf = float(r64[i]);
        r[i] = rf;
        p[i] = rf;
        d[i] = 0.0f;
        red[0] += double(rf) * double(rf);
    }
    grid_reduce_finish<1, kVecThreads>(fin, red, s, 0);
}

// Mixed precision: x += d / scale (FP64), after an inner FP32 solve of
// A d = scale * r.
static __global__ void __launch_bounds__(kVecThreads)
    ir_apply_kernel(int n, double* __restrict__ x, const float* __restrict__ d, const CgState* outer) {
    const double inv = 1.0 / outer->scale;
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads)
        x[i] += double(d[i]) * inv;
}

// ---------------------------------------------------------------------------
// PageRank.
struct PrState {
    double teleport;  // (d * D + 1 - d) / N for the next iteration
    double dangling;  // D of the vector the next iteration reads
    int iter;         // iterations completed
    int pad;
};

// has_out bit j set <=> column j holds an entry <=> vertex j has an out-edge.
static __global__ void __launch_bounds__(kVecThreads)
    mark_columns_kernel(int64_t nnz, const int* __restrict__ col_ind, unsigned* __restrict__ has_out) {
    for (int64_t k = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * kVecThreads) {
        const int c = col_ind[k];
        const unsigned bit = 1u << (c & 31);
        if ((__ldg(has_out + (c >> 5)) & bit) == 0u) atomicOr(has_out + (c >> 5), bit);
    }
}

__device__ __forceinline__ bool is_dangling(const unsigned* has_out, int j) {
    return ((__ldg(has_out + (j >> 5)) >> (j & 31)) & 1u) == 0u;
}

struct FinPrStart {
    PrState* st;
    double damping;
    int n;
    __device__ void finish(const double* tot) const {
        st->dangling = tot[0];
        st->teleport = (damping * tot[0] + (1.0 - damping)) / double(n);
        st->iter = 0;
    }
};

// Optionally x = 1/N; D = sum of x over dangling vertices.
template <class T>
static __global__ void __launch_bounds__(kVecThreads)
    pr_start_kernel(int n, T* __restrict__ x, int init_uniform, const unsigned* __restrict__ has_out,
                    FinPrStart fin, Scratch s) {
    double red[1] = {0.0};
    const T u = T(1.0 / double(n));
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads) {
        T xi;
        if (init_uniform) {
            xi = u;
            x[i] = u;
        } else {
            xi = x[i];
        }
        if (is_dangling(has_out, i)) red[0] += double(xi);
    }
    grid_reduce_finish<1, kVecThreads>(fin, red, s, 0);
}

// y = d (A x) + teleport; L1 += |y - x|; D' += y over dangling rows.
template <class V, class T>
struct OpPageRank {
    using ValT = V;
    using VecT = T;
    using AccT = T;
    using RedT = typename RedOf<T>::type;
    static constexpr int NR = 2;
    static constexpr bool kTwoPhase = true;
    T* __restrict__ y;
    const T* __restrict__ x;
    const unsigned* __restrict__ has_out;
    PrState* st;
    double* l1;  // device, one entry per iteration
    T damping;
    int n;
    T tele;  // set by begin()
    __device__ bool skip() const { return false; }
    // Teleport term, written by the previous launch; read once per thread
    // (every thread reads it before its CTA takes a ticket, and this launch's
    // finish() writes it only after the last ticket).
    __device__ void begin() { tele = T(__ldcg(&st->teleport)); }
    __device__ void row(int r, AccT s, RedT* red) const {
        const T yi = damping * s + tele;
        y[r] = yi;
        red_add_absdiff(red[0], yi, x[r]);
        if (is_dangling(has_out, r)) red_add(red[1], yi);
    }
    __device__ void store(int r, AccT s) const { y[r] = damping * s + tele; }
    __device__ void reduce(int r, RedT* red) const {
        const T yi = __ldcg(y + r);
        red_add_absdiff(red[0], yi, x[r]);
        if (is_dangling(has_out, r)) red_add(red[1], yi);
    }
    __device__ bool reduce4_ok() const { return aligned16(y, x); }
    // Rows r0 .. r0 + 3 (r0 a multiple of 4, y and x 16-byte aligned), in
    // row order, with 16-byte loads and one bitmap word.
    __device__ void reduce4(int r0, RedT* red) const {
        using VT = Vec16<T>;
        constexpr int N = VT::N;
        T yv[4], xv[4];
#pragma unroll
        for (int k = 0; k < 4; k += N) {
            const typename VT::type a = __ldcg(reinterpret_cast<const typename VT::type*>(y + r0 + k));
            const typename VT::type b = __ldg(reinterpret_cast<const typename VT::type*>(x + r0 + k));
#pragma unroll
            for (int e = 0; e < N; ++e) {
                yv[k + e] = VT::get(a, e);
                xv[k + e] = VT::get(b, e);
            }
        }
        const unsigned w = __ldg(has_out + (r0 >> 5)) >> (r0 & 31);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            red_add_absdiff(red[0], yv[k], xv[k]);
            if (((w >> k) & 1u) == 0u) red_add(red[1], yv[k]);
        }
    }
    __device__ void finish(const double* tot) const {
        const int t = st->iter;
        l1[t] = tot[0];
        st->dangling = tot[1];
        st->teleport = (double(damping) * tot[1] + (1.0 - double(damping))) / double(n);
        st->iter = t + 1;
    }
};

}  // namespace lilac
