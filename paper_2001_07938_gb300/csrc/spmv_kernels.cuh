// CSR SpMV kernels, y = A x (the paper's spmv_csr, Section 3.2):
//   y[i] = sum_{row_ptr[i] <= j < row_ptr[i+1]} val[j] * x[col_ind[j]].
//
// Every kernel hands each finished row sum to an epilogue `Op`, which stores
// y (or a fused CG / PageRank / residual update) and may add up to kMaxRed
// FP64 values per row into grid-wide sums.  Grid sums end in the last-CTA
// ticket of lilac_device.cuh, so a launch with reductions needs no second
// kernel, and every sum is taken in an order fixed by the launch shape.
//
// Op concept:
//   using ValT (matrix value type), VecT (x / y type), AccT (row accumulator)
//   static constexpr int NR                 number of FP64 reductions (0..kMaxRed)
//   __device__ bool skip() const            true: the whole launch is a no-op
//   __device__ void begin()                 every thread, once, before any row()
//   using RedT                              per-thread accumulator of the FP64
//                                           sums (double, or CompF32 for FP32)
//   __device__ void row(int r, AccT s, RedT* red) const
//   static constexpr bool kTwoPhase   true: also store(r, s) (writes only) and
//       reduce(r, red) (reads back what store wrote); row() == store + reduce.
//       The MERGE kernel stores while it walks and reduces later, one row per
//       thread, so the walk never waits on the epilogue's loads.
//   __device__ void finish(const double* tot) const   (last CTA, thread 0; NR > 0)
#pragma once

#include <type_traits>

#include "lilac_device.cuh"

namespace lilac {

template <class ValT>
struct CsrView {
    const int* __restrict__ row_ptr;
    const int* __restrict__ col_ind;
    const ValT* __restrict__ val;
    int rows;
};

// One tile of the STAGED kernel.  Row tile: rows [r0, r1) whose nonzeros
// [k0, k1) are contiguous.  Split-row chunk (r1 < 0): nonzeros [k0, k1) of
// split row number r0, written to chunk slot -r1 - 1.
struct TileDesc {
    int r0, r1, k0, k1;
};

struct LongRow {
    int row, first_slot, nchunks, pad;
};

// ---------------------------------------------------------------------------
// SCALAR (V = 1) and VECTOR (V lanes per row) kernels: rows in a grid-stride
// loop straight from global memory; V = 32 is warp-per-row.

template <int V, int THREADS, class Op>
__global__ void __launch_bounds__(THREADS)
    spmv_rows_kernel(CsrView<typename Op::ValT> A, const typename Op::VecT* __restrict__ x,
                     Op op, Scratch s) {
    if (op.skip()) return;
    op.begin();
    using AccT = typename Op::AccT;
    constexpr int NR = Op::NR;
    typename Op::RedT red[NR > 0 ? NR : 1] = {};
    const int lane = threadIdx.x & (V - 1);
    const int group = (int)((blockIdx.x * THREADS + threadIdx.x) / V);
    const int ngroups = (int)(gridDim.x * THREADS / V);
    const unsigned mask = group_mask<V>(threadIdx.x);
    for (int r = group; r < A.rows; r += ngroups) {
        const int kb = A.row_ptr[r], ke = A.row_ptr[r + 1];
        // four independent gathers in flight per lane; the indices and values
        // of the next four are loaded while those gathers are outstanding
        AccT s0 = AccT(0), s1 = AccT(0), s2 = AccT(0), s3 = AccT(0);
        int k = kb + lane;
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        typename Op::ValT v0{}, v1{}, v2{}, v3{};
        if (k + 3 * V < ke) {
            c0 = ld_stream(A.col_ind + k);
            c1 = ld_stream(A.col_ind + k + V);
            c2 = ld_stream(A.col_ind + k + 2 * V);
            c3 = ld_stream(A.col_ind + k + 3 * V);
            v0 = ld_stream(A.val + k);
            v1 = ld_stream(A.val + k + V);
            v2 = ld_stream(A.val + k + 2 * V);
            v3 = ld_stream(A.val + k + 3 * V);
        }
        while (k + 3 * V < ke) {
            const typename Op::VecT x0 = __ldg(x + c0), x1 = __ldg(x + c1);
            const typename Op::VecT x2 = __ldg(x + c2), x3 = __ldg(x + c3);
            const typename Op::ValT w0 = v0, w1 = v1, w2 = v2, w3 = v3;
            const int kn = k + 4 * V;
            if (kn + 3 * V < ke) {
                c0 = ld_stream(A.col_ind + kn);
                c1 = ld_stream(A.col_ind + kn + V);
                c2 = ld_stream(A.col_ind + kn + 2 * V);
                c3 = ld_stream(A.col_ind + kn + 3 * V);
                v0 = ld_stream(A.val + kn);
                v1 = ld_stream(A.val + kn + V);
                v2 = ld_stream(A.val + kn + 2 * V);
                v3 = ld_stream(A.val + kn + 3 * V);
            }
            s0 += AccT(w0) * AccT(x0);
            s1 += AccT(w1) * AccT(x1);
            s2 += AccT(w2) * AccT(x2);
            s3 += AccT(w3) * AccT(x3);
            k = kn;
        }
        {
            // the last (at most three) nonzeros of this lane: loads issued together
            const bool q0 = k < ke, q1 = k + V < ke, q2 = k + 2 * V < ke;
            const int a0 = q0 ? ld_stream(A.col_ind + k) : 0;
            const int a1 = q1 ? ld_stream(A.col_ind + k + V) : 0;
            const int a2 = q2 ? ld_stream(A.col_ind + k + 2 * V) : 0;
            const typename Op::ValT w0 = q0 ? ld_stream(A.val + k) : typename Op::ValT(0);
            const typename Op::ValT w1 = q1 ? ld_stream(A.val + k + V) : typename Op::ValT(0);
            const typename Op::ValT w2 = q2 ? ld_stream(A.val + k + 2 * V) : typename Op::ValT(0);
            if (q0) s0 += AccT(w0) * AccT(__ldg(x + a0));
            if (q1) s1 += AccT(w1) * AccT(__ldg(x + a1));
            if (q2) s2 += AccT(w2) * AccT(__ldg(x + a2));
        }
        AccT sum = (s0 + s1) + (s2 + s3);
        if constexpr (V > 1) sum = group_sum<V>(sum, mask);
        if (lane == 0) op.row(r, sum, red);
    }
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        grid_reduce_finish<NR, THREADS>(op, r2, s, 0);
    }
}

// ---------------------------------------------------------------------------
// STAGED kernel.  Persistent CTAs take tiles blockIdx.x, blockIdx.x + grid,
// ... (static, so the per-CTA sums are reproducible).  Thread 0 streams the
// next tile's val / col_ind / row_ptr segments into the other half of a
// double buffer with cp.async.bulk while the block computes the current one
// from shared memory.  Within a tile, every thread first gathers x for its
// TN / THREADS nonzeros (all loads in flight together) and stores the
// products in shared memory; then groups of V lanes add up one row each.
// Split rows
// (longer than a tile) are summed chunk by chunk; the CTA that adds the last
// chunk (arrival counter) adds the chunk sums in chunk order and runs the
// epilogue for the row.
//
// Shared layout per stage: val[TN + 8] | col[TN + 8] | row_ptr[TR + 8]
// (and one product buffer when the accumulator is wider than the values).
// Copies start at indices rounded down to a multiple of 4 (16 bytes for
// 4- and 8-byte elements) and end rounded up; the device arrays are padded
// by the host so the rounded-up end stays inside the allocation.

template <class ValT, class AccT, int TN, int TR>
struct StagedLayout {
    static constexpr int kValElems = TN + 8;
    static constexpr int kRpElems = TR + 8;
    static constexpr size_t kValBytes = sizeof(ValT) * kValElems;
    static constexpr size_t kColBytes = sizeof(int) * kValElems;
    static constexpr size_t kRpBytes = sizeof(int) * kRpElems;
    static constexpr size_t kStageBytes = kValBytes + kColBytes + kRpBytes;
    // products of a tile: in place over the values, or (value and
    // accumulator types of different size) in one extra buffer
    static constexpr size_t kProdBytes = sizeof(AccT) == sizeof(ValT) ? 0 : sizeof(AccT) * kValElems;
    static constexpr size_t kSmemBytes = 2 * kStageBytes + kProdBytes;
};

template <int V, int THREADS, int TN, int TR, class Op>
__global__ void __launch_bounds__(THREADS)
    spmv_staged_kernel(CsrView<typename Op::ValT> A, const TileDesc* __restrict__ tiles,
                       int ntiles, const LongRow* __restrict__ longs, int nlong,
                       const typename Op::VecT* __restrict__ x, Op op, Scratch s) {
    if (op.skip()) return;
    op.begin();
    using ValT = typename Op::ValT;
    using AccT = typename Op::AccT;
    using L = StagedLayout<ValT, AccT, TN, TR>;
    constexpr int NR = Op::NR;
    constexpr int NGROUPS = THREADS / V;
    constexpr int IPT = TN / THREADS;
    static_assert(TN % THREADS == 0, "tile nonzeros must be a multiple of the block size");

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ TileDesc sdesc[2];
    __shared__ AccT sh_sum[32];
    __shared__ int sh_ok;

    typename Op::RedT red[NR > 0 ? NR : 1] = {};
    const int tid = threadIdx.x;
    const int lane = tid & (V - 1);
    const int group = tid / V;
    const unsigned mask = group_mask<V>(tid);
    const int cnt = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;

    uint64_t policy = 0;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        policy = l2_policy_evict_first();
    }
    __syncthreads();

    auto stage_ptr = [&](int st) { return smem + st * L::kStageBytes; };

    // Thread 0: start the copies of the CTA's i-th tile into stage st.
    auto issue = [&](int i, int st) {
        const TileDesc t = tiles[blockIdx.x + (size_t)i * gridDim.x];
        sdesc[st] = t;
        unsigned char* base = stage_ptr(st);
        const int ka = t.k0 & ~3;
        const int kz = (t.k1 + 3) & ~3;
        const uint32_t nk = (uint32_t)(kz - ka);
        uint32_t bytes = nk * (uint32_t)(sizeof(ValT) + sizeof(int));
        int ra = 0;
        uint32_t nr = 0;
        if (t.r1 >= 0) {
            ra = t.r0 & ~3;
            const int rz = (t.r1 + 1 + 3) & ~3;
            nr = (uint32_t)(rz - ra);
            bytes += nr * (uint32_t)sizeof(int);
        }
        mbar_arrive_expect_tx(&bar[st], bytes);
        if (nk > 0) {
            bulk_g2s(base, A.val + ka, nk * (uint32_t)sizeof(ValT), &bar[st], policy);
            bulk_g2s(base + L::kValBytes, A.col_ind + ka, nk * (uint32_t)sizeof(int), &bar[st],
                     policy);
        }
        if (nr > 0)
            bulk_g2s(base + L::kValBytes + L::kColBytes, A.row_ptr + ra, nr * (uint32_t)sizeof(int),
                     &bar[st], policy);
    };

    // test hook: CTA 0 leaves its first copy unissued (the waits below time
    // out); only this hook is consumed here, another one stays armed
    const bool skip_first = tid == 0 && blockIdx.x == 0 &&
                            atomicCAS(s.status + 1, DEV_INJECT_SKIP_COPY, DEV_INJECT_NONE) ==
                                DEV_INJECT_SKIP_COPY;
    if (cnt > 0 && tid == 0 && !skip_first) issue(0, 0);
    bool failed = false;
    // epilogues with reductions: rows are stored in phase B and reduced one
    // row per thread in the next tile, after its gathers are issued
    constexpr bool kDeferred = Op::kTwoPhase && NR > 0;
    int prev_r0 = 0, prev_n = 0;
    for (int i = 0; i < cnt; ++i) {
        const int st = i & 1;
        if (i + 1 < cnt && tid == 0) {
            fence_proxy_async_smem();
            issue(i + 1, st ^ 1);
        }
        const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)((i >> 1) & 1));
        if (!__syncthreads_and(ok ? 1 : 0)) {
            failed = true;
            // let the other stage's copy (if any) land before leaving
            if (tid == 0 && i + 1 < cnt) (void)mbar_wait_bounded(&bar[st ^ 1], (uint32_t)(((i + 1) >> 1) & 1));
            break;
        }
        const TileDesc t = sdesc[st];
        unsigned char* base = stage_ptr(st);
        const ValT* vs = reinterpret_cast<const ValT*>(base);
        const int* cs = reinterpret_cast<const int*>(base + L::kValBytes);
        const int* rps = reinterpret_cast<const int*>(base + L::kValBytes + L::kColBytes);
        // products overwrite the values in place when the types have one size
        AccT* prod = L::kProdBytes ? reinterpret_cast<AccT*>(smem + 2 * L::kStageBytes)
                                   : reinterpret_cast<AccT*>(base);
        const int ka = t.k0 & ~3;
        const int kb0 = t.k0 - ka, ke0 = t.k1 - ka;
        // Phase A: every thread gathers x for IPT nonzeros of the tile, all
        // loads issued before any is used.
        int cj[IPT];
        typename Op::VecT xj[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int k = kb0 + j * THREADS + tid;
            cj[j] = k < ke0 ? cs[k] : 0;
        }
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int k = kb0 + j * THREADS + tid;
            xj[j] = k < ke0 ? __ldg(x + cj[j]) : typename Op::VecT(0);
        }
        if constexpr (kDeferred) {
            for (int q = tid; q < prev_n; q += THREADS) op.reduce(prev_r0 + q, red);
            prev_n = 0;
        }
        if (t.r1 >= 0) {
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int k = kb0 + j * THREADS + tid;
                if (k < ke0) prod[k] = AccT(vs[k]) * AccT(xj[j]);
            }
            __syncthreads();
            // Phase B: groups of V lanes add each row's products from shared memory.
            const int ra = t.r0 & ~3;
            const int nrows = t.r1 - t.r0;
            for (int rr = group; rr < nrows; rr += NGROUPS) {
                const int kb = rps[t.r0 - ra + rr] - ka;
                const int ke = rps[t.r0 - ra + rr + 1] - ka;
                AccT sum = AccT(0);
                for (int k = kb + lane; k < ke; k += V) sum += prod[k];
                if constexpr (V > 1) sum = group_sum<V>(sum, mask);
                if (lane == 0) {
                    if constexpr (kDeferred)
                        op.store(t.r0 + rr, sum);
                    else
                        op.row(t.r0 + rr, sum, red);
                }
            }
            if constexpr (kDeferred) {
                prev_r0 = t.r0;
                prev_n = nrows;
            }
        } else {
            // chunk of a split row: the whole block sums it
            AccT sum = AccT(0);
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                const int k = kb0 + j * THREADS + tid;
                if (k < ke0) sum += AccT(vs[k]) * AccT(xj[j]);
            }
            sum = block_sum_lead<THREADS, AccT>(sum, sh_sum);
            if (tid == 0) {
                const int lid = t.r0;
                const int slot = -t.r1 - 1;
                s.long_part[slot] = (double)sum;
                __threadfence();
                const LongRow lr = longs[lid];
                const unsigned c = atomicAdd(&s.long_cnt[lid], 1u);
                if (c == (unsigned)lr.nchunks - 1u) {
                    __threadfence();
                    AccT rs = AccT(0);
                    for (int j = 0; j < lr.nchunks; ++j) rs += AccT(__ldcg(&s.long_part[lr.first_slot + j]));
                    typename Op::RedT lred[NR > 0 ? NR : 1] = {};
                    op.row(lr.row, rs, lred);
#pragma unroll
                    for (int q = 0; q < NR; ++q) s.long_red[lid * kMaxRed + q] = red_value(lred[q]);
                    s.long_cnt[lid] = 0u;
                }
            }
        }
        // this thread's shared-memory writes (in-place products) are ordered
        // before the bulk copy that will overwrite the stage
        fence_proxy_async_smem();
        __syncthreads();  // stage st is free for the copy issued in iteration i + 1
    }
    if (failed) {
        if (tid == 0) atomicExch(s.status, DEV_TIMEOUT);
        return;
    }
    if constexpr (kDeferred) {
        for (int q = tid; q < prev_n; q += THREADS) op.reduce(prev_r0 + q, red);
    }
    (void)sh_ok;
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        grid_reduce_finish<NR, THREADS>(op, r2, s, nlong);
    }
}

}  // namespace lilac

namespace lilac {

// Slab s of x, x[c0 .. c0 + w), into shared memory xs[0 .. w), with zeros in
// xs[w .. W] (padding points at W): 16-byte loads when x + c0 is aligned (c0
// is a multiple of 8), eight in flight per thread.
template <int THREADS, class VecT>
__device__ __forceinline__ void slab_load_x(VecT* xs, const VecT* __restrict__ x, int c0, int w,
                                            int W) {
    constexpr int E = 16 / sizeof(VecT);
    const bool al = (reinterpret_cast<uintptr_t>(x + c0) & 15u) == 0;
    const int nv = al ? w / E : 0;
    const uint4* __restrict__ xv = reinterpret_cast<const uint4*>(x + c0);
    uint4* xsv = reinterpret_cast<uint4*>(xs);
    int i = threadIdx.x;
    for (; i + 7 * THREADS < nv; i += 8 * THREADS) {
        uint4 t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = __ldg(xv + i + u * THREADS);
#pragma unroll
        for (int u = 0; u < 8; ++u) xsv[i + u * THREADS] = t[u];
    }
    for (; i < nv; i += THREADS) xsv[i] = __ldg(xv + i);
    for (int j = nv * E + threadIdx.x; j < w; j += THREADS) xs[j] = __ldg(x + c0 + j);
    for (int j = w + threadIdx.x; j <= W; j += THREADS) xs[j] = VecT(0);
}

// ---------------------------------------------------------------------------
// SELL kernels: a sliced ELLPACK copy of the matrix (SELL-C-sigma with C = 32,
// built once per handle in lilac_sell.cu).  Chunk c holds 32 row pieces, one
// per lane, padded to the longest; element k of lane l is at cptr[c] + 32 k + l,
// so every load of a warp is one contiguous segment.  Each lane adds its piece
// with one fused multiply-add per element in nonzero order and no shuffle
// reductions: on GB300 a warp-wide FP64 FMA costs the same issue slot however
// many lanes are active, so FP64 SpMV is bound by FMA issue as much as by HBM,
// and the layout spends (almost) exactly one FMA per nonzero.

// Global-x form.  crow[c * 32 + l] is the lane's row (>= 0), -1 (padding lane)
// or -(2 + p) for piece p of a row longer than the piece cap: its sum goes to
// part[p], and the last of the row's pieces to arrive (counter) adds them in
// piece order (the HUB cold part: its warp adds them in a fixed order) and
// runs the epilogue.
// Padding elements have column -1 (no load; they add 0 * 0).
struct SellView {
    const int* __restrict__ cptr;         // [nchunks + 1]
    const int* __restrict__ crow;         // [nchunks * 32]
    const int* __restrict__ col;          // [cptr[nchunks]]
    const int4* __restrict__ splits;      // per split row {row, first piece, pieces, -}
    const int* __restrict__ piece_split;  // piece -> split row
    int nchunks;
    int nsplit;
    // HUB: the copy holds a row's other (cold) columns only; the slab partials
    // of the slabs q in the row's mask (add_mask per lane, splits[].w for a
    // split row) are added, in slab order, before the epilogue (addP null:
    // none).  They are laid out by lane: addP[q * add_stride + i] for the row
    // of lane i = 32 * chunk + lane, addP[q * add_stride + add_split_base +
    // s] for split row s, so a warp's reads are coalesced.
    const void* addP;
    const uint8_t* add_mask;
    int add_stride;
    int add_split_base;
};

// Slab sums added by a cold lane: those of the first kSellPreSlabs slabs are
// loaded at the start of its chunk, the rest (slab q0 on) here.
#ifndef LILAC_SELL_PRE_SLABS
#define LILAC_SELL_PRE_SLABS 4
#endif
constexpr int kSellPreSlabs = LILAC_SELL_PRE_SLABS;

template <class AccT>
__device__ __forceinline__ AccT sell_add_slabs(const SellView& S, int idx, unsigned mask, AccT acc,
                                               int q0 = 0) {
    const AccT* __restrict__ P = static_cast<const AccT*>(S.addP);
    mask >>= q0;
    for (int q = q0; mask != 0u; ++q, mask >>= 1)
        if (mask & 1u) acc += __ldg(P + (size_t)q * S.add_stride + idx);
    return acc;
}

// Piece p of a split row: its sum goes to part[p], and the last of the row's
// pieces to arrive (counter) adds them in piece order and runs the epilogue.
template <bool kStoreOnly, class AccT, class Op>
__device__ __forceinline__ void sell_finish_piece(const SellView& S, const Op& op, const Scratch& s,
                                                  int p, AccT acc) {
    constexpr int NR = kStoreOnly ? 0 : Op::NR;
    s.long_part[p] = (double)acc;
    __threadfence();
    const int lid = S.piece_split[p];
    const int4 sp = S.splits[lid];
    const unsigned c = atomicAdd(&s.long_cnt[lid], 1u);
    if (c == (unsigned)sp.z - 1u) {
        __threadfence();
        AccT rs = AccT(0);
        for (int j = 0; j < sp.z; ++j) rs += AccT(__ldcg(&s.long_part[sp.y + j]));
        if (S.addP) rs = sell_add_slabs(S, S.add_split_base + lid, (unsigned)sp.w, rs);
        if constexpr (kStoreOnly) {
            op.store(sp.x, rs);
        } else {
            typename Op::RedT lred[NR > 0 ? NR : 1] = {};
            op.row(sp.x, rs, lred);
#pragma unroll
            for (int q = 0; q < NR; ++q) s.long_red[lid * kMaxRed + q] = red_value(lred[q]);
        }
        s.long_cnt[lid] = 0u;
        __threadfence();  // the epilogue sums before this CTA's grid-reduction ticket
    }
}

// The same for the whole warp (warp-uniform call; the FP32 HUB cold part,
// whose hub rows split into hundreds of pieces): every lane holding a piece stores
// its sum to part[p] and takes a ticket on its row's counter; for each lane
// whose piece came last, the warp adds the row's pieces -- lane l the pieces
// l, l + 32, ... in order, then a butterfly of shuffles, the same fixed order
// for a given piece count -- and that lane runs the epilogue: a few L2 round
// trips instead of one per few pieces.  (It costs registers: the other SELL
// forms, whose split rows have few pieces, keep the one-lane finish.)
template <bool kStoreOnly, class AccT, class Op>
__device__ __forceinline__ void sell_finish_pieces(const SellView& S, const Op& op, const Scratch& s,
                                                   int who, AccT acc, int lane) {
    constexpr int NR = kStoreOnly ? 0 : Op::NR;
    bool last = false;
    int4 sp = make_int4(0, 0, 0, 0);
    int lid = 0;
    if (who < -1) {
        const int p = -who - 2;
        s.long_part[p] = (double)acc;
        __threadfence();
        lid = S.piece_split[p];
        sp = S.splits[lid];
        last = atomicAdd(&s.long_cnt[lid], 1u) == (unsigned)sp.z - 1u;
    }
    unsigned m = __ballot_sync(0xffffffffu, last);
    if (m == 0u) return;
    __threadfence();
    while (m != 0u) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const int first = __shfl_sync(0xffffffffu, sp.y, src);
        const int np = __shfl_sync(0xffffffffu, sp.z, src);
        AccT v = AccT(0);
        for (int j = lane; j < np; j += 32) v += AccT(__ldcg(&s.long_part[first + j]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == src) {
            AccT rs = v;
            if (S.addP) rs = sell_add_slabs(S, S.add_split_base + lid, (unsigned)sp.w, rs);
            if constexpr (kStoreOnly) {
                op.store(sp.x, rs);
            } else {
                typename Op::RedT lred[NR > 0 ? NR : 1] = {};
                op.row(sp.x, rs, lred);
#pragma unroll
                for (int q = 0; q < NR; ++q) s.long_red[lid * kMaxRed + q] = red_value(lred[q]);
            }
            s.long_cnt[lid] = 0u;
            __threadfence();  // the epilogue sums before this CTA's grid-reduction ticket
        }
    }
}

// kStoreOnly (two-phase epilogues): rows are only stored; the reductions run
// in row order in rows_reduce_kernel, which keeps their loads coalesced when
// the rows are sorted by length.
// kAdd (the cold part of a HUB copy): every lane adds its row's slab sums
// (S.addP), loaded at the start of its chunk.
// The HUB cold part's lanes are short (a few elements each): with FP32
// vectors the kernel is bound by load latency, so it is held to 48 registers
// for five CTAs per SM (80 registers gave two: 1.13x slower on an R-MAT
// scale-22 PageRank); FP64 forms would spill there and keep their registers.
// The other forms keep the compiler's own choice (0: no minimum; a minimum
// of 1 let it take up to 96 registers and cost the FP32 Poisson CG SpMV 14%).
#ifndef LILAC_HUB_COLD_MIN_BLOCKS
#define LILAC_HUB_COLD_MIN_BLOCKS 5
#endif
template <class Op, bool kAdd>
constexpr int sell_min_blocks() {
    return kAdd && sizeof(typename Op::VecT) == 4 ? LILAC_HUB_COLD_MIN_BLOCKS : 0;
}
template <int THREADS, int UNR, bool kStoreOnly, class Op, bool kAdd = false>
__global__ void __launch_bounds__(THREADS, sell_min_blocks<Op, kAdd>())
    spmv_sell_kernel(SellView S, const typename Op::ValT* __restrict__ val,
                     const typename Op::VecT* __restrict__ x, Op op, Scratch s) {
    if (op.skip()) return;
    op.begin();
    using ValT = typename Op::ValT;
    using VecT = typename Op::VecT;
    using AccT = typename Op::AccT;
    constexpr int NR = kStoreOnly ? 0 : Op::NR;
    typename Op::RedT red[NR > 0 ? NR : 1] = {};
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)(gridDim.x * (THREADS / 32));
    // the next chunk's offsets and lane row are loaded while this chunk runs:
    // short chunks (many on power-law matrices) then cost no extra round trip
    int ch = (int)((blockIdx.x * THREADS + threadIdx.x) >> 5);
    int nbase = 0, nend = 0, nwho = -1;
    unsigned nmask = 0u;  // slab sums to add (HUB cold part), also loaded ahead
    if (ch < S.nchunks) {
        nbase = __ldg(S.cptr + ch);
        nend = __ldg(S.cptr + ch + 1);
        nwho = __ldg(S.crow + (size_t)ch * 32 + lane);
        if constexpr (kAdd) nmask = __ldg(S.add_mask + (size_t)ch * 32 + lane);
    }
    for (; ch < S.nchunks; ch += nwarps) {
        const int base = nbase;
        const int width = (nend - base) >> 5;
        const int who = nwho;
        const unsigned mask = who >= 0 ? nmask : 0u;
        if (ch + nwarps < S.nchunks) {
            nbase = __ldg(S.cptr + ch + nwarps);
            nend = __ldg(S.cptr + ch + nwarps + 1);
            nwho = __ldg(S.crow + (size_t)(ch + nwarps) * 32 + lane);
            if constexpr (kAdd) nmask = __ldg(S.add_mask + (size_t)(ch + nwarps) * 32 + lane);
        }
        // the row's slab sums of the first kSellPreSlabs slabs, issued before
        // the element loop (added after it, in slab order)
        AccT pre[kAdd && kSellPreSlabs > 0 ? kSellPreSlabs : 1];
        if constexpr (kAdd) {
#pragma unroll
            for (int q = 0; q < kSellPreSlabs; ++q)
                pre[q] = (mask >> q) & 1u ? __ldg(static_cast<const AccT*>(S.addP) +
                                                   (size_t)q * S.add_stride + (size_t)ch * 32 + lane)
                                          : AccT(0);
        }
        const ValT* __restrict__ vp = val + base + lane;
        const int* __restrict__ cp = S.col + base + lane;
        AccT acc = AccT(0);
        int k = 0;
        for (; k + UNR <= width; k += UNR) {
            ValT vv[UNR];
            int cc[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                vv[u] = ld_stream(vp + 32 * (k + u));
                cc[u] = ld_stream(cp + 32 * (k + u));
            }
            VecT xx[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) xx[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : VecT(0);
#pragma unroll
            for (int u = 0; u < UNR; ++u) acc += AccT(vv[u]) * AccT(xx[u]);
        }
        if (k < width) {
            // the last (fewer than UNR) elements, loads issued together; the
            // bound is the same for the whole warp, so skipped FMAs cost nothing
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
            for (int u = 0; u < UNR; ++u) xx[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : VecT(0);
#pragma unroll
            for (int u = 0; u < UNR; ++u)
                if (k + u < width) acc += AccT(vv[u]) * AccT(xx[u]);
        }
        if (who >= 0) {
            if constexpr (kAdd) {
                if (mask != 0u) {
#pragma unroll
                    for (int q = 0; q < kSellPreSlabs; ++q)
                        if ((mask >> q) & 1u) acc += pre[q];
                    if (mask >> kSellPreSlabs)
                        acc = sell_add_slabs(S, ch * 32 + lane, mask, acc, kSellPreSlabs);
                }
            }
            if constexpr (kStoreOnly)
                op.store(who, acc);
            else
                op.row(who, acc, red);
        }
        if constexpr (kAdd && sizeof(VecT) == 4) {
            if (__any_sync(0xffffffffu, who < -1))
                sell_finish_pieces<kStoreOnly, AccT>(S, op, s, who, acc, lane);
        } else if (who < -1) {
            sell_finish_piece<kStoreOnly, AccT>(S, op, s, -who - 2, acc);
        }
    }
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        grid_reduce_finish<NR, THREADS>(op, r2, s, S.nsplit);
    }
}

// Second phase of a two-phase epilogue: op.reduce for every row, in row order,
// then the grid sum.  An op with reduce4 (PageRank) takes four consecutive
// rows per step with 16-byte loads when its vectors allow (reduce4_ok)
// (one 4-byte load per row kept the pass at a quarter of HBM bandwidth).
template <class Op, class = void>
struct HasReduce4 : std::false_type {};
template <class Op>
struct HasReduce4<Op, std::void_t<decltype(&Op::reduce4)>> : std::true_type {};

template <int THREADS, class Op>
__global__ void __launch_bounds__(THREADS) rows_reduce_kernel(int rows, Op op, Scratch s) {
    if (op.skip()) return;
    op.begin();
    constexpr int NR = Op::NR;
    typename Op::RedT red[NR > 0 ? NR : 1] = {};
    const int t0 = blockIdx.x * THREADS + threadIdx.x, G = gridDim.x * THREADS;
    int r1 = 0;  // rows before r1 are done by reduce4
    if constexpr (HasReduce4<Op>::value) {
        if (op.reduce4_ok()) {
            const int nq = rows / 4;
            for (int q = t0; q < nq; q += G) op.reduce4(4 * q, red);
            r1 = 4 * nq;
        }
    }
    for (int r = r1 + t0; r < rows; r += G) op.reduce(r, red);
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        grid_reduce_finish<NR, THREADS>(op, r2, s, 0);
    }
}

// ---------------------------------------------------------------------------
// SLAB kernel: the sliced ELL layout over column slabs, x read from shared
// memory.  Random 8-byte gathers through L1 cost one tag lookup per distinct
// line (about one per cycle per SM); from shared memory they cost one bank
// access each.  The columns are cut into S slabs of W columns (x slab of at
// most kSlabMaxBytes) and the rows into G groups of about equal nonzero
// count.  Each (slab, group) pair holds the pieces of the group's rows (the
// nonzeros whose column lies in the slab, in CSR order, 16-bit local
// columns) as sliced ELL chunks sorted by piece length.  One CTA of THREADS
// threads per (slab, group), one per SM, loads slab s of x into shared memory
// (plus a zero at index W that padding points to) and runs the pair's chunks,
// warps taking chunks from a shared counter; a lane's piece sum goes to
// P[s][row].  The last of the group's S CTAs to finish (arrival counter) adds
// P over the slabs in slab order for every row of the group and runs the
// epilogue; its reductions go to partial slot g, summed in slot order.
#ifndef LILAC_SLAB_PIPE
#define LILAC_SLAB_PIPE 0
#endif
constexpr bool kSlabPipe = LILAC_SLAB_PIPE != 0;

struct SlabView {
    const int* __restrict__ cptr;    // [S * chunks + 1]
    const int* __restrict__ crow;    // [chunks * 32]: row, or -1 (padding lane)
    const uint16_t* __restrict__ col;
    const int4* __restrict__ ctas;   // {slab, first chunk, end chunk, group}
    const int2* __restrict__ groups; // [G] rows [r0, r1)
    unsigned* __restrict__ gcnt;     // [G] arrival counters (zero between launches)
    int rows, ncols, W, S, G;
};

// The piece sum of one lane of chunk `ch`: one FMA per element in element
// order, UNR elements (value, 16-bit column, x from shared memory) in flight.
// PIPE: the loads of the next UNR elements are issued before the FMAs of the
// current ones, so a warp keeps loads in flight while it waits for the FP64
// pipe.
template <int UNR, bool PIPE, class AccT, class ValT, class VecT>
__device__ __forceinline__ AccT slab_lane_sum(const SlabView& V, const ValT* __restrict__ sval,
                                              const VecT* xs, int base, int width, int lane);

template <int UNR, bool PIPE, class AccT, class ValT, class VecT>
__device__ __forceinline__ AccT slab_chunk_sum(const SlabView& V, const ValT* __restrict__ sval,
                                               const VecT* xs, int ch, int lane) {
    const int base = __ldg(V.cptr + ch);
    const int width = (__ldg(V.cptr + ch + 1) - base) >> 5;
    return slab_lane_sum<UNR, PIPE, AccT>(V, sval, xs, base, width, lane);
}

// The same with the chunk's element offset and width given (loaded ahead).
template <int UNR, bool PIPE, class AccT, class ValT, class VecT>
__device__ __forceinline__ AccT slab_lane_sum(const SlabView& V, const ValT* __restrict__ sval,
                                              const VecT* xs, int base, int width, int lane) {
    const ValT* __restrict__ vp = sval + base + lane;
    const uint16_t* __restrict__ cp = V.col + base + lane;
    AccT acc = AccT(0);
    if constexpr (PIPE) {
        ValT va[UNR];
        int ca[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const bool q = u < width;
            va[u] = q ? ld_stream(vp + 32 * u) : ValT(0);
            ca[u] = q ? (int)ld_stream(cp + 32 * u) : V.W;
        }
        for (int k = 0; k < width; k += UNR) {
            ValT vb[UNR];
            int cb[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const bool q = k + UNR + u < width;
                vb[u] = q ? ld_stream(vp + 32 * (k + UNR + u)) : ValT(0);
                cb[u] = q ? (int)ld_stream(cp + 32 * (k + UNR + u)) : V.W;
            }
            if (k + UNR <= width) {
#pragma unroll
                for (int u = 0; u < UNR; ++u) acc += AccT(va[u]) * AccT(xs[ca[u]]);
            } else {
                // the bound is the same for the whole warp: skipped FMAs cost nothing
#pragma unroll
                for (int u = 0; u < UNR; ++u)
                    if (k + u < width) acc += AccT(va[u]) * AccT(xs[ca[u]]);
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                va[u] = vb[u];
                ca[u] = cb[u];
            }
        }
        return acc;
    }
    int k = 0;
    for (; k + UNR <= width; k += UNR) {
        ValT vv[UNR];
        int cc[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            vv[u] = ld_stream(vp + 32 * (k + u));
            cc[u] = ld_stream(cp + 32 * (k + u));
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) acc += AccT(vv[u]) * AccT(xs[cc[u]]);
    }
    if (k < width) {
        // the last (fewer than UNR) elements, loads issued together; the
        // bound is the same for the whole warp, so skipped FMAs cost nothing
        ValT vv[UNR];
        int cc[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const bool q = k + u < width;
            vv[u] = q ? ld_stream(vp + 32 * (k + u)) : ValT(0);
            cc[u] = q ? (int)ld_stream(cp + 32 * (k + u)) : V.W;
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (k + u < width) acc += AccT(vv[u]) * AccT(xs[cc[u]]);
    }
    return acc;
}

template <int THREADS, int UNR, class Op>
__global__ void __launch_bounds__(THREADS, 1)
    spmv_slab_kernel(SlabView V, const typename Op::ValT* __restrict__ sval,
                     const typename Op::VecT* __restrict__ x, typename Op::AccT* __restrict__ P,
                     Op op, Scratch s) {
    if (op.skip()) return;
    op.begin();
    using VecT = typename Op::VecT;
    using AccT = typename Op::AccT;
    constexpr int NR = Op::NR;
    extern __shared__ __align__(16) unsigned char slab_smem[];
    __shared__ int next_chunk;
    __shared__ int last_of_group;
    VecT* xs = reinterpret_cast<VecT*>(slab_smem);
    const int4 c = V.ctas[blockIdx.x];  // {slab, first chunk, end chunk, group}
    const int sl = c.x;
    const int c0 = sl * V.W;
    slab_load_x<THREADS>(xs, x, c0, min(V.W, V.ncols - c0), V.W);
    if (threadIdx.x == 0) next_chunk = c.y + THREADS / 32;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    AccT* __restrict__ Ps = P + (size_t)sl * V.rows;
    int ch = c.y + (int)(threadIdx.x >> 5);
    while (ch < c.z) {
        const int row = __ldg(V.crow + (size_t)ch * 32 + lane);
        const AccT acc = slab_chunk_sum<UNR, kSlabPipe, AccT>(V, sval, xs, ch, lane);
        if (row >= 0) Ps[row] = acc;
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&next_chunk, 1);
        ch = __shfl_sync(0xffffffffu, nx, 0);
    }
    // the last CTA of the row group combines the slabs and runs the epilogue
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
        last_of_group = atomicAdd(&V.gcnt[c.w], 1u) == (unsigned)(V.S - 1) ? 1 : 0;
    __syncthreads();
    const bool last = last_of_group != 0;
    typename Op::RedT red[NR > 0 ? NR : 1] = {};
    if (last) {
        __threadfence();
        const int2 gr = V.groups[c.w];
        for (int r = gr.x + (int)threadIdx.x; r < gr.y; r += THREADS) {
            AccT sum = __ldcg(P + r);
            for (int q = 1; q < V.S; ++q) sum += __ldcg(P + (size_t)q * V.rows + r);
            op.row(r, sum, red);
        }
        if (threadIdx.x == 0) V.gcnt[c.w] = 0u;
    }
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        grid_reduce_slots<NR, THREADS>(op, r2, s, last ? c.w : -1, V.G);
    }
}

// ---------------------------------------------------------------------------
// HUB kernels (lilac_hub.cu builds the copies).  A power-law matrix whose x
// is far larger than L1 spends its time on random x gathers that each move a
// 32-byte sector from L2 for a 4- or 8-byte value.  The hub columns, the most
// frequent ones, hold most of the nonzeros: their x is gathered once per
// SpMV (hub_gather_kernel), cut into S slabs of W values, and held in shared
// memory by one CTA per SM (hub_pieces_kernel), which sums every row's piece
// of that slab with 16-bit slab-local columns into P[s][row] (rows without a
// piece in the slab are no lane of it), laid out by the row's lane in the
// cold copy.  The other (cold) nonzeros form a sliced ELL copy run by
// spmv_sell_kernel, which adds the partials of the slabs in the row's mask to
// its sum before the epilogue.  Each element issues one load, from shared
// memory or through L1/L2, never both.

// x of the hub columns (hot[h], h < H) into xhot, ahead of the pieces kernel.
template <class VecT>
__global__ void hub_gather_kernel(int H, const int* __restrict__ hot, const VecT* __restrict__ x,
                                  VecT* __restrict__ xhot) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x)
        xhot[h] = __ldg(x + __ldg(hot + h));
}

// Hot pieces longer than the copy's cap are cut into sub-pieces of at most
// the cap, one lane each (lane row -(2 + sub-piece)): sub-piece p's sum goes
// to part[p], and the last of a split's sub-pieces to arrive (counter) adds
// them in order into P[slab][row].
struct HubSplits {
    const int4* __restrict__ splits;  // {row, first sub-piece, sub-pieces, slab}
    const int* __restrict__ sub_split;  // sub-piece -> split
    double* part;
    unsigned* cnt;
};

// One CTA per {slab, first chunk, end chunk} run: slab s of xhot in shared
// memory (plus a zero at W for padding), warps take the run's chunks from a
// shared counter, lane l of a chunk stores its piece sum to P[s][pos], pos
// (the lane's crow entry, V.rows the stride of P) the row's place in the
// cold copy.
template <int THREADS, int UNR, class Op>
__global__ void __launch_bounds__(THREADS, 1)
    hub_pieces_kernel(SlabView V, const int4* __restrict__ ranges,
                      const typename Op::ValT* __restrict__ hval,
                      const typename Op::VecT* __restrict__ xhot, int H,
                      typename Op::AccT* __restrict__ P, HubSplits hs, Op op) {
    if (op.skip()) return;
    using VecT = typename Op::VecT;
    using AccT = typename Op::AccT;
    extern __shared__ __align__(16) unsigned char hub_smem[];
    __shared__ int next_chunk;
    VecT* xs = reinterpret_cast<VecT*>(hub_smem);
    const int4 c = ranges[blockIdx.x];  // {slab, first chunk, end chunk, -}
    const int c0 = c.x * V.W;
    slab_load_x<THREADS>(xs, xhot, c0, min(V.W, H - c0), V.W);
    if (threadIdx.x == 0) next_chunk = c.y + THREADS / 32;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    AccT* __restrict__ Ps = P + (size_t)c.x * V.rows;
    // the next chunk is taken, and its offsets and lane rows loaded, while
    // this one runs: short chunks then cost no extra round trip
    int ch = c.y + (int)(threadIdx.x >> 5);
    int nbase = 0, nend = 0, nrow = -1;
    if (ch < c.z) {
        nbase = __ldg(V.cptr + ch);
        nend = __ldg(V.cptr + ch + 1);
        nrow = __ldg(V.crow + (size_t)ch * 32 + lane);
    }
    while (ch < c.z) {
        const int row = nrow, base = nbase, width = (nend - nbase) >> 5;
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&next_chunk, 1);
        const int nch = __shfl_sync(0xffffffffu, nx, 0);
        if (nch < c.z) {
            nbase = __ldg(V.cptr + nch);
            nend = __ldg(V.cptr + nch + 1);
            nrow = __ldg(V.crow + (size_t)nch * 32 + lane);
        }
        const AccT acc = slab_lane_sum<UNR, false, AccT>(V, hval, xs, base, width, lane);
        if (row >= 0) {
            Ps[row] = acc;
        } else if (row < -1) {
            const int sp = -row - 2;
            hs.part[sp] = (double)acc;
            __threadfence();
            const int lid = __ldg(hs.sub_split + sp);
            const int4 q = hs.splits[lid];
            if (atomicAdd(&hs.cnt[lid], 1u) == (unsigned)q.z - 1u) {
                __threadfence();
                AccT sum = AccT(0);
                for (int j = 0; j < q.z; ++j) sum += AccT(__ldcg(&hs.part[q.y + j]));
                P[(size_t)q.w * V.rows + q.x] = sum;
                hs.cnt[lid] = 0u;
            }
        }
        ch = nch;
    }
}

// ---------------------------------------------------------------------------
// JDS kernel (jagged diagonal storage, Section 3.2): slot s holds the s-th
// longest row (row slot_row[s], len[s] nonzeros); jagged diagonal d stores
// the d-th nonzero of every slot with len > d, contiguously by slot.  One
// thread per slot: consecutive threads read consecutive entries of each
// diagonal (coalesced), and the threads of a warp have about the same row
// length.  A row's products are added in nonzero order.
template <int THREADS, class Op>
__global__ void __launch_bounds__(THREADS)
    spmv_jds_kernel(int rows, const int* __restrict__ slot_row, const int* __restrict__ len,
                    const int* __restrict__ jd_ptr, const int* __restrict__ col,
                    const typename Op::ValT* __restrict__ val,
                    const typename Op::VecT* __restrict__ x, Op op, Scratch s) {
    if (op.skip()) return;
    op.begin();
    using AccT = typename Op::AccT;
    constexpr int NR = Op::NR;
    typename Op::RedT red[NR > 0 ? NR : 1] = {};
    for (int sl = blockIdx.x * THREADS + threadIdx.x; sl < rows; sl += gridDim.x * THREADS) {
        const int L = __ldg(len + sl);
        AccT sum = AccT(0);
#pragma unroll 4
        for (int d = 0; d < L; ++d) {
            const int k = __ldg(jd_ptr + d) + sl;
            sum += AccT(ld_stream(val + k)) * AccT(__ldg(x + ld_stream(col + k)));
        }
        op.row(__ldg(slot_row + sl), sum, red);
    }
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        grid_reduce_finish<NR, THREADS>(op, r2, s, 0);
    }
}

}  // namespace lilac

namespace lilac {

// ---------------------------------------------------------------------------
// MERGE kernel: merge-path partition (Merrill & Garland, "Merge-based
// parallel sparse matrix-vector multiplication", SC 2016).  The merge of the
// row-end list (row_ptr[1..rows]) with the nonzero indices (0..nnz-1) has
// rows + nnz items; CTA c takes items [c*P, (c+1)*P), so every CTA gets the
// same mix of row ends and nonzeros whatever the row lengths.  A CTA walks
// its items in sub-tiles of ITEMS: the products of the sub-tile's nonzeros go
// to shared memory, then every thread takes ITEMS/THREADS consecutive path
// items (its start found by a merge-path search in shared memory) and walks
// them in order: a nonzero adds its product to the running row sum, a row end
// closes the row.  A row that starts before the thread's first item (the
// thread's first closed row, or the row still open at its end) gets the
// pieces of the earlier threads through a segmented scan keyed by row, so a
// row of any length costs the same per item as a short one.  A row still open
// at the end of a sub-tile carries its sum to the next one.
// Across CTAs, each CTA records a head piece (its first row, which is open
// at the CTA's start, if it ends in this CTA) and a tail piece (the row
// open at its end); the last CTA to finish adds, for each row that crosses
// CTAs, the tail pieces and the closing head piece in CTA order, and runs
// the epilogue for it.
struct MergeCarry {
    int head_row;  // -1: none
    int tail_row;  // -1: none
    double head_v;
    double tail_v;
};

// Path point d: (i, j) with i + j = d, i = row ends consumed, j = nonzeros
// consumed; a nonzero j is consumed before the end of row i when j < row_ptr[i+1].
__device__ __forceinline__ int2 merge_path_search(int64_t d, const int* __restrict__ row_ptr,
                                                  int rows, int64_t nnz) {
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < rows ? d : rows;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(row_ptr + mid + 1) <= d - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    return make_int2((int)lo, (int)(d - lo));
}

// The MERGE kernel runs in little shared memory (~17 KB per CTA with FP32
// sums, ~25 KB with FP64), which leaves most of the unified L1 / shared array
// to L1: the x gathers in flight need it (a large shared carveout measured at
// half the speed on a random-column graph).  Plain stores keep a full SM of
// CTAs resident (2048 threads, 32 registers).
#ifndef LILAC_MERGE_RED_THREADS_PER_SM
#define LILAC_MERGE_RED_THREADS_PER_SM 1024
#endif
template <class Op, int THREADS>
constexpr int merge_min_blocks() {
    // epilogues with reductions keep more values live (the deferred
    // reductions overlap the next gathers): half an SM of threads with up to
    // 64 registers each measured faster than a full SM with spills
    return (Op::NR > 0 ? LILAC_MERGE_RED_THREADS_PER_SM : 2048) / THREADS;
}

template <int THREADS, int ITEMS, class Op>
__global__ void __launch_bounds__(THREADS, merge_min_blocks<Op, THREADS>())
    spmv_merge_kernel(CsrView<typename Op::ValT> A, int64_t nnz, const int2* __restrict__ coords,
                      int64_t per_cta, const typename Op::VecT* __restrict__ x, Op op,
                      double* __restrict__ partials, MergeCarry* __restrict__ carries,
                      unsigned* __restrict__ ticket) {
    using AccT = typename Op::AccT;
    constexpr int NR = Op::NR;
    constexpr int IPT = ITEMS / THREADS;
    constexpr int NWARPS = THREADS / 32;
    static_assert(ITEMS % THREADS == 0 && THREADS % 32 == 0,
                  "items per sub-tile must be a multiple of the block size, a multiple of 32");
    if (op.skip()) return;
    op.begin();

    __shared__ int rp_s[ITEMS + 2];
    __shared__ AccT prod_s[ITEMS];
    __shared__ int w_key[NWARPS];
    __shared__ AccT w_val[NWARPS];
    // path point, carried row sum and head flag at the start of a sub-tile,
    // double-buffered by sub-tile parity (one barrier per sub-tile hands over)
    __shared__ int s_i[2], s_j[2], s_head_pending[2];
    __shared__ AccT s_running[2];
    __shared__ int s_head_row;
    __shared__ AccT s_head_v;
    __shared__ double sh_red[kMaxRed * 32];
    __shared__ int am_last;

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int rows = A.rows;
    const int64_t total = (int64_t)rows + nnz;
    const int64_t D0 = (int64_t)blockIdx.x * per_cta;
    const int64_t D1 = D0 + per_cta < total ? D0 + per_cta : total;
    typename Op::RedT red[NR > 0 ? NR : 1] = {};

    if (tid == 0) {
        int2 st = make_int2(rows, (int)nnz);
        if (D0 < total) st = coords ? coords[blockIdx.x] : merge_path_search(D0, A.row_ptr, rows, nnz);
        s_i[0] = st.x;
        s_j[0] = st.y;
        // the row open at the CTA's start is the previous CTA's tail: its
        // piece here always goes through the carries
        s_head_pending[0] = (blockIdx.x > 0 && D0 < total && st.x < rows) ? 1 : 0;
        s_running[0] = AccT(0);
        s_head_row = -1;
        s_head_v = AccT(0);
    }
    __syncthreads();
    constexpr bool kDeferred = Op::kTwoPhase && NR > 0;
    constexpr int RPT = (ITEMS + 2 + THREADS - 1) / THREADS;
    // rows closed by the previous sub-tile whose reductions are still due
    int prev_i = 0, prev_n = 0, prev_head = 0;
    int p = 0;
    for (int64_t d = D0; d < D1; d += ITEMS, p ^= 1) {
        const int len = (int)(D1 - d < ITEMS ? D1 - d : ITEMS);
        const int i = s_i[p], j = s_j[p];
        const AccT running = s_running[p];
        const int head_pending = s_head_pending[p];
        // row_ptr[i .. i + nrw): the sub-tile closes at most `len` rows
        const int nrw = min(ITEMS + 2, rows + 1 - i);
        // (with deferred reductions the row_ptr loads stay in registers until
        // the gathers are issued; otherwise they go straight to shared memory,
        // which needs fewer registers)
        int rv[kDeferred ? RPT : 1];
        if constexpr (kDeferred) {
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int t = q * THREADS + tid;
                rv[q] = t < nrw ? __ldg(A.row_ptr + i + t) : 0;
            }
        } else {
            for (int t = tid; t < nrw; t += THREADS) rp_s[t] = __ldg(A.row_ptr + i + t);
        }
        // products of nonzeros [j, jz): the sub-tile holds at most `len` of them
        const int jz = (int)min((int64_t)j + len, nnz);
        int cj[IPT];
        typename Op::VecT xj[IPT];
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int k = j + q * THREADS + tid;
            cj[q] = k < jz ? ld_stream(A.col_ind + k) : 0;
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int k = j + q * THREADS + tid;
            xj[q] = k < jz ? __ldg(x + cj[q]) : typename Op::VecT(0);
        }
        if constexpr (kDeferred) {
            // reductions of the rows the previous sub-tile closed: their loads
            // overlap this sub-tile's gathers
            for (int q = tid; q < prev_n; q += THREADS)
                if (q > 0 || !prev_head) op.reduce(prev_i + q, red);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int t = q * THREADS + tid;
                if (t < nrw) rp_s[t] = rv[q];
            }
        }
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int k = j + q * THREADS + tid;
            if (k < jz) prod_s[k - j] = AccT(ld_stream(A.val + k)) * AccT(xj[q]);
        }
        __syncthreads();
        // this thread's path items [o0, o1) of the sub-tile; its start point
        // (r, k), r + k = d + o0, by a merge-path search in shared memory
        const int o0 = min(tid * IPT, len), o1 = min(o0 + IPT, len);
        int r, k;
        {
            const int64_t dd = d + o0;
            int64_t lo = dd - nnz > i ? dd - nnz : i;
            int64_t hi = dd - j < rows ? dd - j : rows;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if ((int64_t)rp_s[mid + 1 - i] <= dd - mid - 1)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            r = (int)lo;
            k = (int)(dd - lo);
        }
        // walk: rows closed after the first one are complete here; the first
        // (row r at the start) waits for the earlier threads' pieces
        AccT acc = AccT(0), first_v = AccT(0);
        int first_r = -1;
        for (int o = o0; o < o1; ++o) {
            if (k < rp_s[r + 1 - i]) {
                acc += prod_s[k - j];
                ++k;
            } else {
                if (first_r < 0) {
                    first_r = r;
                    first_v = acc;
                } else if constexpr (Op::kTwoPhase) {
                    op.store(r, acc);
                } else {
                    op.row(r, acc, red);
                }
                acc = AccT(0);
                ++r;
            }
        }
        // inclusive segmented scan of the open-row pieces, keyed by row (keys
        // do not decrease with the thread index): within the warp ...
        const int key = r;
        AccT v = acc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const AccT vu = __shfl_up_sync(0xffffffffu, v, off);
            const int ku = __shfl_up_sync(0xffffffffu, key, off);
            if (lane >= off && ku == key) v += vu;
        }
        if (lane == 31) {
            w_key[warp] = key;
            w_val[warp] = v;
        }
        __syncthreads();
        // ... then across the earlier warps' totals
        AccT pre = AccT(0);
        int pre_key = -1;
        for (int w = 0; w < warp; ++w) {
            const int kw = w_key[w];
            pre = kw == pre_key ? pre + w_val[w] : w_val[w];
            pre_key = kw;
        }
        const AccT full = (warp > 0 && key == pre_key) ? v + pre : v;
        // pieces of row r before this thread = the previous thread's scan
        const AccT up = __shfl_up_sync(0xffffffffu, full, 1);
        const AccT incoming = lane > 0 ? up : (warp > 0 ? pre : AccT(0));
        if (first_r >= 0) {
            AccT sum = incoming + first_v;
            if (first_r == i) sum = running + sum;
            if (first_r == i && head_pending) {
                s_head_row = i;
                s_head_v = sum;
            } else if constexpr (Op::kTwoPhase) {
                op.store(first_r, sum);
            } else {
                op.row(first_r, sum, red);
            }
        }
        if (tid == THREADS - 1) {
            // the last thread ends where the sub-tile ends
            s_i[p ^ 1] = r;
            s_j[p ^ 1] = k;
            s_running[p ^ 1] = r == i ? running + full : full;
            s_head_pending[p ^ 1] = r > i ? 0 : head_pending;
        }
        __syncthreads();
        if constexpr (kDeferred) {
            // the reductions over the rows closed here, [i, ie), run in the next
            // sub-tile (or below), consecutive rows on consecutive threads; the
            // barrier made the stores visible.  The CTA's open first row is
            // finished from the carries instead.
            prev_i = i;
            prev_n = s_i[p ^ 1] - i;
            prev_head = head_pending;
        }
    }
    if constexpr (kDeferred) {
        for (int q = tid; q < prev_n; q += THREADS)
            if (q > 0 || !prev_head) op.reduce(prev_i + q, red);
    }
    // publish carries and partial sums; the last CTA fixes up and finishes
    double tot[NR > 0 ? NR : 1];
    if constexpr (NR > 0) {
        double r2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) r2[q] = red_value(red[q]);
        block_sum<NR, THREADS>(r2, tot, sh_red);
    }
    if (tid == 0) {
        MergeCarry mc;
        mc.head_row = s_head_row;
        mc.head_v = (double)s_head_v;
        const bool open_tail = D0 < total && s_i[p] < rows;
        mc.tail_row = open_tail ? s_i[p] : -1;
        mc.tail_v = open_tail ? (double)s_running[p] : 0.0;
        carries[blockIdx.x] = mc;
#pragma unroll
        for (int q = 0; q < NR; ++q) partials[blockIdx.x * NR + q] = tot[q];
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int G = (int)gridDim.x;
    typename Op::RedT fred[NR > 0 ? NR : 1] = {};
    for (int c = tid; c < G; c += THREADS) {
        const int r = __ldcg(&carries[c].tail_row);
        if (r < 0 || (c > 0 && __ldcg(&carries[c - 1].tail_row) == r)) continue;
        // this CTA holds the first piece of row r: add the later pieces in order
        AccT v = AccT(__ldcg(&carries[c].tail_v));
        for (int k = c + 1; k < G; ++k) {
            if (__ldcg(&carries[k].head_row) == r) {
                v += AccT(__ldcg(&carries[k].head_v));
                break;
            }
            if (__ldcg(&carries[k].tail_row) != r) break;
            v += AccT(__ldcg(&carries[k].tail_v));
        }
        op.row(r, v, fred);
    }
    if constexpr (NR > 0) {
        double acc[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = red_value(fred[q]);
        for (int c = tid; c < G; c += THREADS) {
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] += __ldcg(&partials[c * NR + q]);
        }
        block_sum<NR, THREADS>(acc, tot, sh_red);
        if (tid == 0) op.finish(tot);
    }
    if (tid == 0) *ticket = 0u;
}

}  // namespace lilac
