// Batched kernels: many CSR problems of uneven size in one persistent launch.
//
// The work list holds (problem, tile) items for the SpMV phases and
// (problem, chunk) items for the vector phases of CG; persistent CTAs take
// items blockIdx.x, blockIdx.x + grid, ...  Every reduction of a problem is
// kept per item (partial sums per tile or chunk) and added, in item order,
// by the CTA that completes the problem's last item (arrival counter), so a
// problem's result depends only on its own tiling -- the same alone and in
// any mix.
//
// CG problems run in one of two precisions: FP64 (values, vectors and sums),
// or FP32 CG with FP64 reliable updates (FP32 values, vectors and row sums,
// FP64 dot products, solution accumulated in FP64 and the residual replaced
// by the FP64 b - A x whenever the FP32 residual fell by delta; the same
// method as lilac_cg precision 2).
#pragma once

#include "ops.cuh"

namespace lilac {

enum BatchKind : int { BK_SPMV = 0, BK_CG = 1 };
enum BatchPrec : int { BP_F64 = 0, BP_F32_RU = 2 };
// How a problem's SpMV is cut into work items: the handle's STAGED tiles, or
// groups of chunks of its sliced ELL copy (the layout the handle's tuner
// picked for SELL and SLAB matrices).
enum BatchLayout : int { BL_TILES = 0, BL_SELL = 1 };

constexpr int kBatchThreads = 256;
constexpr int kBatchItems = 2048;   // nonzeros per tile: matches the STAGED tile list
constexpr int kBatchRows = 1024;    // rows per tile: matches the STAGED tile list
#ifndef LILAC_BATCH_SPMV_CTAS
#define LILAC_BATCH_SPMV_CTAS 4
#endif
constexpr int kBatchSpmvCtasPerSm = LILAC_BATCH_SPMV_CTAS;  // register bound of the SpMV-phase kernel
constexpr int kBatchChunk = 1024;   // vector elements per chunk item (4 per thread)
constexpr int kBatchSellChunks = kBatchThreads / 32;  // SELL chunks per item (one per warp)

struct BatchProb {
    // matrix (a handle's arrays and STAGED tile list, or its SELL copy)
    const int* row_ptr;
    const int* col_ind;
    const double* val;   // FP64 values (FP64 handles; null for FP32 handles)
    const float* val32;  // FP32 values: the handle's own (FP32 handles) or its FP32 copy
    const TileDesc* tiles;
    const LongRow* longs;
    // split rows: STAGED chunk sums / SELL piece sums, arrival counters and
    // epilogue sums (per problem, in its workspace)
    double* long_part;
    unsigned* long_cnt;
    double* long_red;
    int rows;
    int ntiles;  // SpMV-phase items: tiles (BL_TILES) or chunk groups (BL_SELL)
    int nlong;   // split rows
    int kind;
    int nchunks;
    int prec;
    int layout;
    int f32;     // 1: FP32 handle (FP32 values; SpMV vectors x_in / y_out are float)
    // BL_SELL: the handle's sliced ELL copy (values of the handle's type)
    const int* scptr;
    const int* scrow;
    const int* scol;
    const void* sval;
    const int4* ssplits;
    const int* spiece_split;
    int snchunks;
    int spad;
    // SpMV: y = A x (double, or float for FP32 handles)
    const void* x_in;
    void* y_out;
    // CG: b, x (FP64); r, p, q (FP64) or r32, p32, q32 and the FP32 correction d32
    const double* b;
    double* x;
    double* r;
    double* p;
    double* q;
    float* r32;
    float* p32;
    float* q32;
    float* d32;
    CgState* st;
    double rtol;
    double delta2;  // BP_F32_RU: replace when r.r <= delta2 * r.r at the last replacement
    int max_iter;
    int pad;
    // per-item partial sums: [0, 2 ntiles) SpMV phases (two per tile), then
    // one per vector chunk; arrival counters of the SpMV and vector phases
    double* part;
    unsigned* cnt;
};

struct BatchItem {
    int prob;
    int idx;
};

// Sum of a problem's NR-wide partials (item i at part + i * stride) and its
// split-row sums (extra + i * kMaxRed), by the whole block of the item that
// arrived last: thread t adds items t, t + THREADS, ... in order, then the
// block's fixed tree -- an order set by the problem's item count alone, so a
// problem's sums do not depend on the other problems of the batch.  The
// result is valid in thread 0.
template <int NR, int THREADS>
__device__ __forceinline__ void batch_sum_parts(const double* part, int n, int stride,
                                                const double* extra, int nextra,
                                                double (&out)[NR], double* sh) {
    double acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < n; i += THREADS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] += __ldcg(part + (size_t)i * stride + q);
    }
    for (int i = threadIdx.x; i < nextra; i += THREADS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] += __ldcg(extra + (size_t)i * kMaxRed + q);
    }
    block_sum<NR, THREADS>(acc, out, sh);
}

__device__ __forceinline__ bool batch_ru_due(const CgState* st) {
    return *reinterpret_cast<const volatile int*>(&st->update) != 0 && !cg_done(st);
}

// Epilogues of the batched SpMV phases (row r's sum s; up to two FP64 sums).
template <class T>
struct BEpiStore {  // y = A x
    T* y;
    __device__ void row(int r, T s, double*) const { y[r] = s; }
};
template <class T>
struct BEpiPq {  // q = A p, p.q
    T* q;
    const T* p;
    __device__ void row(int r, T s, double* red) const {
        q[r] = s;
        red[0] += double(p[r]) * double(s);
    }
};
struct BEpiResid {  // r32 = float(b - A x), ||b - A x||^2, float(r).float(r)
    float* r32;
    const double* b;
    __device__ void row(int r, double s, double* red) const {
        const double ri = b[r] - s;
        const float rf = float(ri);
        r32[r] = rf;
        red[0] += ri * ri;
        red[1] += double(rf) * double(rf);
    }
};

// Rows of a staged tile by groups of V lanes: lane l of a group adds
// elements l, l + V, ... of its row (one FMA each), then the group's tree.
template <int V, class AccT, class Epi>
__device__ __forceinline__ void batch_tile_rows(const TileDesc& t, int nrows, const AccT* vs,
                                                const AccT* xs, const int* rp_s, const Epi& epi,
                                                double* red) {
    constexpr int NGROUPS = kBatchThreads / V;
    const int tid = threadIdx.x;
    const int lane = tid & (V - 1), group = tid / V;
    const unsigned mask = group_mask<V>(tid);
    for (int rr = group; rr < nrows; rr += NGROUPS) {
        const int kb = rp_s[rr] - t.k0, ke = rp_s[rr + 1] - t.k0;
        AccT sum = AccT(0);
        for (int k = kb + lane; k < ke; k += V) sum = fma(vs[k], xs[k], sum);
        sum = group_sum<V>(sum, mask);
        if (lane == 0) epi.row(t.r0 + rr, sum, red);
    }
}

// One tile of one problem: its values and gathered x to shared memory (one
// coalesced pass), then rows by groups of V lanes -- 4 for short rows, 16
// when the tile's rows average 48 elements or more, so that every lane has
// a few elements of a row -- with one FMA per element; a chunk of a split
// row is summed by the block and finished by the chunk that arrives last.
// Returns the tile's FP64 sums in red[0..1].
template <class ValT, class VecT, class AccT, class Epi>
__device__ __forceinline__ void batch_tile(const BatchProb& P, const TileDesc& t,
                                           const ValT* __restrict__ val,
                                           const VecT* __restrict__ xin, const Epi& epi,
                                           double* red, unsigned char* smem, int* rp_s,
                                           AccT* sh) {
    constexpr int THREADS = kBatchThreads;
    constexpr int IPT = kBatchItems / THREADS;
    AccT* vs = reinterpret_cast<AccT*>(smem);
    AccT* xs = vs + kBatchItems;
    const int tid = threadIdx.x;
    int cj[IPT];
    ValT vj[IPT];
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int k = t.k0 + j * THREADS + tid;
        cj[j] = k < t.k1 ? ld_stream(P.col_ind + k) : 0;
        vj[j] = k < t.k1 ? ld_stream(val + k) : ValT(0);
    }
#pragma unroll
    for (int j = 0; j < IPT; ++j) {
        const int k = t.k0 + j * THREADS + tid;
        if (k < t.k1) {
            vs[j * THREADS + tid] = AccT(vj[j]);
            xs[j * THREADS + tid] = AccT(__ldg(xin + cj[j]));
        }
    }
    if (t.r1 >= 0) {
        const int nrows = t.r1 - t.r0;
        for (int q = tid; q <= nrows; q += THREADS) rp_s[q] = __ldg(P.row_ptr + t.r0 + q);
        __syncthreads();
        if (t.k1 - t.k0 >= 48 * nrows)  // uniform over the block
            batch_tile_rows<16>(t, nrows, vs, xs, rp_s, epi, red);
        else
            batch_tile_rows<4>(t, nrows, vs, xs, rp_s, epi, red);
    } else {
        __syncthreads();
        AccT sum = AccT(0);
        for (int k = tid; k < t.k1 - t.k0; k += THREADS) sum = fma(vs[k], xs[k], sum);
        sum = block_sum_lead<THREADS, AccT>(sum, sh);
        if (tid == 0) {
            const int lid = t.r0, slot = -t.r1 - 1;
            P.long_part[slot] = double(sum);
            __threadfence();
            const LongRow lr = P.longs[lid];
            if (atomicAdd(&P.long_cnt[lid], 1u) == (unsigned)lr.nchunks - 1u) {
                __threadfence();
                AccT rs = AccT(0);
                for (int j = 0; j < lr.nchunks; ++j) rs += AccT(__ldcg(&P.long_part[lr.first_slot + j]));
                double lred[2] = {0.0, 0.0};
                epi.row(lr.row, rs, lred);
                P.long_red[lid * kMaxRed] = lred[0];
                P.long_red[lid * kMaxRed + 1] = lred[1];
                P.long_cnt[lid] = 0u;
            }
        }
    }
}

// One chunk group of a problem's sliced ELL copy (BL_SELL): warp w sums chunk
// kBatchSellChunks * idx + w the way spmv_sell_kernel does (one lane per row
// or piece, one FMA per element in element order, padding column -1).  A
// lane holding a whole row runs the epilogue; a piece of a split row goes to
// its slot, and the last piece to arrive adds the pieces in piece order and
// runs the epilogue (its sums to long_red).  The group's FP64 sums are left
// in red[0..1] of every thread.
template <class ValT, class VecT, class AccT, class Epi>
__device__ __forceinline__ void batch_sell_item(const BatchProb& P, int idx,
                                                const ValT* __restrict__ val,
                                                const VecT* __restrict__ xin, const Epi& epi,
                                                double* red) {
    constexpr int UNR = 8;
    const int lane = threadIdx.x & 31;
    const int ch = idx * kBatchSellChunks + (int)(threadIdx.x >> 5);
    if (ch >= P.snchunks) return;
    const int base = __ldg(P.scptr + ch);
    const int width = (__ldg(P.scptr + ch + 1) - base) >> 5;
    const int who = __ldg(P.scrow + (size_t)ch * 32 + lane);
    const ValT* __restrict__ vp = val + base + lane;
    const int* __restrict__ cp = P.scol + base + lane;
    AccT acc = AccT(0);
    for (int k = 0; k < width; k += UNR) {
        ValT vv[UNR];
        int cc[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const bool q = k + u < width;
            vv[u] = q ? ld_stream(vp + 32 * (k + u)) : ValT(0);
            cc[u] = q ? ld_stream(cp + 32 * (k + u)) : -1;
        }
        VecT xx[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) xx[u] = cc[u] >= 0 ? __ldg(xin + cc[u]) : VecT(0);
        if (k + UNR <= width) {
#pragma unroll
            for (int u = 0; u < UNR; ++u) acc += AccT(vv[u]) * AccT(xx[u]);
        } else {
            // the bound is the same for the whole warp: skipped FMAs cost nothing
#pragma unroll
            for (int u = 0; u < UNR; ++u)
                if (k + u < width) acc += AccT(vv[u]) * AccT(xx[u]);
        }
    }
    if (who >= 0) {
        epi.row(who, acc, red);
    } else if (who < -1) {
        const int p = -who - 2;
        P.long_part[p] = double(acc);
        __threadfence();
        const int lid = __ldg(P.spiece_split + p);
        const int4 sp = P.ssplits[lid];
        if (atomicAdd(&P.long_cnt[lid], 1u) == (unsigned)sp.z - 1u) {
            __threadfence();
            AccT rs = AccT(0);
            for (int j = 0; j < sp.z; ++j) rs += AccT(__ldcg(&P.long_part[sp.y + j]));
            double lred[2] = {0.0, 0.0};
            epi.row(sp.x, rs, lred);
            P.long_red[lid * kMaxRed] = lred[0];
            P.long_red[lid * kMaxRed + 1] = lred[1];
            P.long_cnt[lid] = 0u;
        }
    }
}

// One SpMV-phase item of a problem in its layout.
template <class ValT, class VecT, class AccT, class Epi>
__device__ __forceinline__ void batch_item(const BatchProb& P, int idx, const ValT* __restrict__ val,
                                           const ValT* __restrict__ sval,
                                           const VecT* __restrict__ xin, const Epi& epi,
                                           double* red, unsigned char* smem, int* rp_s, AccT* sh) {
    if (P.layout == BL_SELL)
        batch_sell_item<ValT, VecT, AccT>(P, idx, sval, xin, epi, red);
    else
        batch_tile<ValT, VecT, AccT>(P, P.tiles[idx], val, xin, epi, red, smem, rp_s, sh);
}

// Problem-level ends of the SpMV phases (last tile of the problem, thread 0,
// given the problem's sums).
__device__ __forceinline__ void batch_finish_pq(const BatchProb& P, double pq) {
    CgState* st = P.st;
    st->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
        st->status = LILAC_ERR_BREAKDOWN;
        st->done = 1;
    } else {
        st->alpha = st->rr / pq;
    }
}

__device__ __forceinline__ void batch_finish_resid(const BatchProb& P, double rr_true, double rr32) {
    CgState* st = P.st;
    st->true_rr = rr_true;
    st->updates += 1;
    st->update = 0;
    if (rr_true == 0.0 || (st->tol2 >= 0.0 && rr_true <= st->tol2)) {
        st->done = 1;
        st->status = LILAC_OK;
    } else if (st->iters >= st->max_iter) {
        st->done = 1;
        st->status = st->tol2 >= 0.0 ? LILAC_ERR_NOT_CONVERGED : LILAC_OK;
    } else {
        st->beta = rr32 / st->rr;  // r.r before this iteration
        st->rr = rr32;
        st->rr_anchor = rr32;
    }
}

// SpMV phases.  MODE 0: y = A x (BK_SPMV) or q = A p with p.q -> alpha (BK_CG,
// in the problem's precision).  MODE 1: the FP64 residual of BP_F32_RU
// problems whose replacement is due (other items return at once).
template <int MODE>
static __global__ void __launch_bounds__(kBatchThreads, kBatchSpmvCtasPerSm)
    batch_spmv_kernel(const BatchProb* __restrict__ probs, const BatchItem* __restrict__ items,
                      const int* __restrict__ nitems_dev) {
    constexpr int THREADS = kBatchThreads;
    __shared__ __align__(16) unsigned char smem[2 * kBatchItems * sizeof(double)];
    __shared__ int rp_s[kBatchRows + 2];
    __shared__ double sh[32];
    __shared__ float shf[32];
    __shared__ double shr[kMaxRed * 32];
    __shared__ int last;
    const int tid = threadIdx.x;
    const int nitems = *nitems_dev;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const BatchProb& P = probs[item.prob];
        const int kind = P.kind;
        // uniform over the block: flags change only in earlier launches
        if (MODE == 0 && kind == BK_CG && cg_done(P.st)) continue;
        if (MODE == 1 && !(kind == BK_CG && P.prec == BP_F32_RU && batch_ru_due(P.st))) continue;
        double red[2] = {0.0, 0.0};
        const float* sv32 = static_cast<const float*>(P.sval);
        const double* sv64 = static_cast<const double*>(P.sval);
        if (MODE == 1) {
            // FP64 residual b - A x with the handle's values (FP32 ones promoted)
            if (P.f32)
                batch_item<float, double, double>(P, item.idx, P.val32, sv32, P.x,
                                                  BEpiResid{P.r32, P.b}, red, smem, rp_s, sh);
            else
                batch_item<double, double, double>(P, item.idx, P.val, sv64, P.x,
                                                   BEpiResid{P.r32, P.b}, red, smem, rp_s, sh);
        } else if (kind == BK_SPMV) {
            if (P.f32)
                batch_item<float, float, float>(P, item.idx, P.val32, sv32,
                                                static_cast<const float*>(P.x_in),
                                                BEpiStore<float>{static_cast<float*>(P.y_out)}, red,
                                                smem, rp_s, shf);
            else
                batch_item<double, double, double>(P, item.idx, P.val, sv64,
                                                   static_cast<const double*>(P.x_in),
                                                   BEpiStore<double>{static_cast<double*>(P.y_out)},
                                                   red, smem, rp_s, sh);
        } else if (P.prec == BP_F32_RU) {
            batch_item<float, float, float>(P, item.idx, P.val32, sv32, P.p32,
                                            BEpiPq<float>{P.q32, P.p32}, red, smem, rp_s, shf);
        } else {
            batch_item<double, double, double>(P, item.idx, P.val, sv64, P.p,
                                               BEpiPq<double>{P.q, P.p}, red, smem, rp_s, sh);
        }
        if (kind == BK_CG) {
            // this tile's share of the sums; the problem's last tile finishes
            double tot[2];
            block_sum<2, THREADS>(red, tot, shr);
            if (tid == 0) {
                P.part[2 * item.idx] = tot[0];
                P.part[2 * item.idx + 1] = tot[1];
                __threadfence();
                last = atomicAdd(&P.cnt[0], 1u) == (unsigned)P.ntiles - 1u;
            }
            __syncthreads();
            if (last) {  // uniform over the block
                __threadfence();
                double sums[2];
                batch_sum_parts<2, THREADS>(P.part, P.ntiles, 2, P.long_red, P.nlong, sums, shr);
                if (tid == 0) {
                    if (MODE == 0)
                        batch_finish_pq(P, sums[0]);
                    else
                        batch_finish_resid(P, sums[0], sums[1]);
                    P.cnt[0] = 0u;
                }
            }
        }
        __syncthreads();
    }
}

// Vector phases of CG over (problem, chunk) items.
//   PHASE 0: start      x = 0, r = p = b (d = 0), r.r
//   PHASE 1: update     x (or d) += alpha p, r -= alpha q, r.r -> beta, convergence
//                       (BP_F32_RU: or flag a residual replacement)
//   PHASE 2: direction  p = r + beta p
//   PHASE 3: BP_F32_RU problems with a replacement due: x += d (FP64), d = 0
template <int PHASE>
static __global__ void __launch_bounds__(kBatchThreads)
    batch_vec_kernel(const BatchProb* __restrict__ probs, const BatchItem* __restrict__ items,
                     const int* __restrict__ nitems_dev) {
    constexpr int THREADS = kBatchThreads;
    __shared__ double shr[kMaxRed * 32];
    __shared__ int last;
    const int tid = threadIdx.x;
    const int nitems = *nitems_dev;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem item = items[it];
        const BatchProb& P = probs[item.prob];
        CgState* st = P.st;
        const bool ru = P.prec == BP_F32_RU;
        if (PHASE != 0 && cg_done(st)) continue;  // uniform over the block
        if (PHASE == 3 && !(ru && batch_ru_due(st))) continue;
        const int i0 = item.idx * kBatchChunk;
        const int i1 = min(P.rows, i0 + kBatchChunk);
        double red = 0.0;
        if (PHASE == 0) {
            for (int i = i0 + tid; i < i1; i += THREADS) {
                const double bi = P.b[i];
                P.x[i] = 0.0;
                if (ru) {
                    const float bf = float(bi);
                    P.r32[i] = bf;
                    P.p32[i] = bf;
                    P.d32[i] = 0.0f;
                    red += double(bf) * double(bf);
                } else {
                    P.r[i] = bi;
                    P.p[i] = bi;
                    red += bi * bi;
                }
            }
        } else if (PHASE == 1) {
            if (ru) {
                const float alpha = float(st->alpha);
                for (int i = i0 + tid; i < i1; i += THREADS) {
                    P.d32[i] += alpha * P.p32[i];
                    const float ri = P.r32[i] - alpha * P.q32[i];
                    P.r32[i] = ri;
                    red += double(ri) * double(ri);
                }
            } else {
                const double alpha = st->alpha;
                for (int i = i0 + tid; i < i1; i += THREADS) {
                    P.x[i] += alpha * P.p[i];
                    const double ri = P.r[i] - alpha * P.q[i];
                    P.r[i] = ri;
                    red += ri * ri;
                }
            }
        } else if (PHASE == 2) {
            if (ru) {
                const float beta = float(st->beta);
                for (int i = i0 + tid; i < i1; i += THREADS) P.p32[i] = P.r32[i] + beta * P.p32[i];
            } else {
                const double beta = st->beta;
                for (int i = i0 + tid; i < i1; i += THREADS) P.p[i] = P.r[i] + beta * P.p[i];
            }
            continue;  // no reduction
        } else {
            for (int i = i0 + tid; i < i1; i += THREADS) {
                P.x[i] += double(P.d32[i]);
                P.d32[i] = 0.0f;
            }
            continue;  // no reduction
        }
        double r1[1] = {red}, tot[1];
        block_sum<1, THREADS>(r1, tot, shr);
        double* vpart = P.part + 2 * (size_t)P.ntiles;
        if (tid == 0) {
            vpart[item.idx] = tot[0];
            __threadfence();
            last = atomicAdd(&P.cnt[1], 1u) == (unsigned)P.nchunks - 1u;
        }
        __syncthreads();
        if (last) {  // uniform over the block
            __threadfence();
            double sum[1];
            batch_sum_parts<1, THREADS>(vpart, P.nchunks, 1, nullptr, 0, sum, shr);
            if (tid == 0) {
                const double s = sum[0];
                if (PHASE == 0) {
                    st->rr = s;
                    st->bb = s;
                    st->tol2 = P.rtol > 0.0 ? P.rtol * P.rtol * s : -1.0;
                    st->iters = 0;
                    st->max_iter = P.max_iter;
                    st->done = s == 0.0 ? 1 : 0;
                    st->status = s == 0.0 ? LILAC_OK : LILAC_ERR_NOT_CONVERGED;
                    st->rr_anchor = s;
                    st->delta2 = P.delta2;
                    st->update = 0;
                    st->updates = 0;
                    st->true_rr = -1.0;
                } else {
                    const int iters = st->iters + 1;
                    st->iters = iters;
                    if (ru) {
                        if (s <= st->delta2 * st->rr_anchor || s == 0.0 ||
                            (st->tol2 >= 0.0 && s <= st->tol2) || iters >= st->max_iter) {
                            st->update = 1;  // st->rr keeps the previous r.r for beta
                        } else {
                            st->beta = s / st->rr;
                            st->rr = s;
                        }
                    } else {
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
                }
                P.cnt[1] = 0u;
            }
        }
        __syncthreads();
    }
}

}  // namespace lilac
