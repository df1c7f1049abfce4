// SpMV launch dispatch: the handle's variant and lanes-per-row select one
// instantiation of the kernels in spmv_kernels.cuh.  Grids are persistent:
// the SM count times the resident CTAs per SM, never more CTAs than there
// is work.
#pragma once

#include "lilac_impl.h"

namespace lilac {

template <class Kernel>
int occupancy_per_sm(Kernel k, int threads, size_t smem) {
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        bps = 1;
    }
    return bps < 1 ? 1 : bps;
}

// Resident CTAs per SM of one kernel instantiation, per device (0: unknown).
template <int V, class Op, bool STAGED>
int& bps_slot(int device) {
    static int cache[64] = {};
    return cache[device & 63];
}

// The first use of an instantiation on a device queries its occupancy (and
// raises its shared-memory limit); prepare_spmv() does that ahead of a
// stream capture, where such calls must not happen.
template <int V, class Op>
lilac_status prepare_rows(lilac_csr_s* A) {
    int& bps = bps_slot<V, Op, false>(A->device);
    if (bps == 0) {
        auto kern = spmv_rows_kernel<V, kRowsThreads, Op>;
        // no shared memory: give the unified L1 / shared array to L1, which
        // caches the gathered x
        LILAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        bps = occupancy_per_sm(kern, kRowsThreads, 0);
    }
    return LILAC_OK;
}

template <int V, class Op>
lilac_status prepare_staged(lilac_csr_s* A) {
    using L = StagedLayout<typename Op::ValT, typename Op::AccT, kTileNnz, kTileRows>;
    int& bps = bps_slot<V, Op, true>(A->device);
    if (bps == 0) {
        auto kern = spmv_staged_kernel<V, kStagedThreads, kTileNnz, kTileRows, Op>;
        LILAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)L::kSmemBytes));
        bps = occupancy_per_sm(kern, kStagedThreads, L::kSmemBytes);
    }
    return LILAC_OK;
}

template <int V, class Op>
lilac_status launch_rows(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                         const Op& op, cudaStream_t stream) {
    LILAC_TRY(prepare_rows<V, Op>(A));
    const int bps = bps_slot<V, Op, false>(A->device);
    const int64_t need = ((int64_t)A->rows * V + kRowsThreads - 1) / kRowsThreads;
    int64_t grid = (int64_t)A->sm_count * bps;
    if (grid > need) grid = need;
    if (grid > kMaxCtas) grid = kMaxCtas;
    if (grid < 1) grid = 1;
    CsrView<typename Op::ValT> view{A->row_ptr.as<int>(), A->col_ind.as<int>(), val, A->rows};
    spmv_rows_kernel<V, kRowsThreads, Op>
        <<<(unsigned)grid, kRowsThreads, 0, stream>>>(view, x, op, A->scratch());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

template <int V, class Op>
lilac_status launch_staged(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                           const Op& op, cudaStream_t stream) {
    using L = StagedLayout<typename Op::ValT, typename Op::AccT, kTileNnz, kTileRows>;
    if (A->ntiles == 0 && Op::NR == 0) return LILAC_OK;  // no rows and nothing to sum
    LILAC_TRY(prepare_staged<V, Op>(A));
    const int bps = bps_slot<V, Op, true>(A->device);
    int64_t grid = (int64_t)A->sm_count * bps;
    if (grid > A->ntiles) grid = A->ntiles;
    if (grid > kMaxCtas) grid = kMaxCtas;
    if (grid < 1) grid = 1;
    CsrView<typename Op::ValT> view{A->row_ptr.as<int>(), A->col_ind.as<int>(), val, A->rows};
    spmv_staged_kernel<V, kStagedThreads, kTileNnz, kTileRows, Op>
        <<<(unsigned)grid, kStagedThreads, L::kSmemBytes, stream>>>(
            view, A->tiles.as<TileDesc>(), A->ntiles, A->longs.as<LongRow>(), A->nlong, x, op,
            A->scratch());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// Resident CTAs per SM of a MERGE instantiation.  No shared-memory carveout
// is requested: the driver then sizes shared memory to what the resident CTAs
// use and leaves the rest to L1 (a larger carveout starves the x gathers in
// flight, measured at half the speed on a random-column graph).
template <class Kernel>
int merge_setup(Kernel kern) {
    return occupancy_per_sm(kern, kMergeThreads, 0);
}

template <int V, class Op>
lilac_status prepare_merge(lilac_csr_s* A) {
    int& bps = bps_slot<V + 128, Op, false>(A->device);
    if (bps == 0) bps = merge_setup(spmv_merge_kernel<kMergeThreads, kMergeItems, Op>);
    return LILAC_OK;
}

template <int V, class Op>
lilac_status launch_merge(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                          const Op& op, cudaStream_t stream) {
    LILAC_TRY(prepare_merge<V, Op>(A));
    CsrView<typename Op::ValT> view{A->row_ptr.as<int>(), A->col_ind.as<int>(), val, A->rows};
    spmv_merge_kernel<kMergeThreads, kMergeItems, Op><<<(unsigned)A->merge_grid, kMergeThreads, 0, stream>>>(
        view, A->nnz, A->merge_coords.as<int2>(), A->merge_per_cta, x, op, A->partials.as<double>(),
        A->merge_carries.as<MergeCarry>(), A->ticket.as<unsigned>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// JDS: the copy holds the handle's own values; another value array (an FP32
// copy) goes to STAGED, as does a handle whose copy is not built.
template <int V, class Op>
lilac_status prepare_jds(lilac_csr_s* A) {
    int& bps = bps_slot<V + 192, Op, false>(A->device);
    if (bps == 0) {
        auto kern = spmv_jds_kernel<kRowsThreads, Op>;
        LILAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        bps = occupancy_per_sm(kern, kRowsThreads, 0);
    }
    return prepare_staged<V, Op>(A);
}

template <int V, class Op>
lilac_status launch_jds(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                        const Op& op, cudaStream_t stream) {
    if (!A->jds_built || (const void*)val != A->val.p) return launch_staged<V, Op>(A, val, x, op, stream);
    LILAC_TRY(prepare_jds<V, Op>(A));
    const int bps = bps_slot<V + 192, Op, false>(A->device);
    int64_t grid = (int64_t)A->sm_count * bps;
    const int64_t need = ((int64_t)A->rows + kRowsThreads - 1) / kRowsThreads;
    if (grid > need) grid = need;
    if (grid > kMaxCtas) grid = kMaxCtas;
    if (grid < 1) grid = 1;
    spmv_jds_kernel<kRowsThreads, Op><<<(unsigned)grid, kRowsThreads, 0, stream>>>(
        A->rows, A->jds_slot_row.as<int>(), A->jds_len.as<int>(), A->jds_ptr.as<int>(),
        A->jds_col.as<int>(), A->jds_val.as<typename Op::ValT>(), x, op, A->scratch());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// STAGED at the handle's lanes per row: where a copy-based variant (SLAB,
// SELL) falls back, vector_width keeps the STAGED width to use.
template <class Op>
lilac_status prepare_staged_any(lilac_csr_s* A) {
    switch (A->vwidth) {
        case 1: return prepare_staged<1, Op>(A);
        case 2: return prepare_staged<2, Op>(A);
        case 4: return prepare_staged<4, Op>(A);
        case 8: return prepare_staged<8, Op>(A);
        case 16: return prepare_staged<16, Op>(A);
        default: return prepare_staged<32, Op>(A);
    }
}

template <class Op>
lilac_status launch_staged_any(lilac_csr_s* A, const typename Op::ValT* val,
                               const typename Op::VecT* x, const Op& op, cudaStream_t stream) {
    switch (A->vwidth) {
        case 1: return launch_staged<1, Op>(A, val, x, op, stream);
        case 2: return launch_staged<2, Op>(A, val, x, op, stream);
        case 4: return launch_staged<4, Op>(A, val, x, op, stream);
        case 8: return launch_staged<8, Op>(A, val, x, op, stream);
        case 16: return launch_staged<16, Op>(A, val, x, op, stream);
        default: return launch_staged<32, Op>(A, val, x, op, stream);
    }
}

// Elements in flight per lane in the sliced ELL kernels (SELL, SLAB).
#ifndef LILAC_SELL_UNROLL
#define LILAC_SELL_UNROLL 8
#endif
constexpr int kSellUnroll = LILAC_SELL_UNROLL;
#ifndef LILAC_SLAB_UNROLL
#define LILAC_SLAB_UNROLL 4
#endif
constexpr int kSlabUnroll = LILAC_SLAB_UNROLL;
// Elements in flight per lane in the HUB pieces kernel (FP32 values and
// 16-bit columns: more of them fit in a lane's registers than SLAB's).
#ifndef LILAC_HUB_UNROLL
#define LILAC_HUB_UNROLL 16
#endif
constexpr int kHubUnroll = LILAC_HUB_UNROLL;

// SLAB: one CTA per SM holding a slab of x in shared memory (lilac_sell.cu
// builds the sliced ELL copy of every slab and row group).  The copy holds the
// handle's own values; another value array (an FP32 copy) goes to STAGED, as
// does a handle without a copy.
template <int V, class Op>
lilac_status prepare_slab(lilac_csr_s* A) {
    int& bps = bps_slot<V + 64, Op, true>(A->device);
    if (bps == 0) {
        auto kern = spmv_slab_kernel<kSlabThreads, kSlabUnroll, Op>;
        LILAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSlabMaxBytes + 64));
        bps = 1;
    }
    return LILAC_OK;
}

template <int V, class Op>
lilac_status launch_slab(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                         const Op& op, cudaStream_t stream) {
    if (!A->slab_built || (const void*)val != A->val.p) return launch_staged_any<Op>(A, val, x, op, stream);
    LILAC_TRY(prepare_slab<V, Op>(A));
    // the slab and the zero after it, in 16-byte units
    const size_t smem = (sizeof(typename Op::VecT) * ((size_t)A->slab_W + 1) + 15) & ~size_t(15);
    SlabView view{A->slab_cptr.as<int>(), A->slab_crow.as<int>(), A->slab_col.as<uint16_t>(),
                  A->slab_ctas.as<int4>(), A->slab_groups.as<int2>(), A->slab_gcnt.as<unsigned>(),
                  A->rows, A->ncols, A->slab_W, A->slab_S, A->slab_G};
    spmv_slab_kernel<kSlabThreads, kSlabUnroll, Op><<<(unsigned)A->slab_grid, kSlabThreads, smem, stream>>>(
        view, A->slab_val.as<typename Op::ValT>(), x, A->slab_P.as<typename Op::AccT>(), op,
        A->scratch());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// SLAB, CG form (FP64 q = A p with p.q; spmv_slab_cg_kernel): runs when the
// handle's SLAB copy holds the values being multiplied.
inline bool slab_cg_active(const lilac_csr_s* A, const void* val) {
    return A->variant == LILAC_VARIANT_SLAB && A->slab_built && val == A->val.p &&
           A->dtype == LILAC_F64 && A->slab_pq.p != nullptr && A->rows == A->ncols;
}

inline lilac_status prepare_slab_cg(lilac_csr_s* A) {
    static int done[64] = {};
    if (!done[A->device & 63]) {
        auto kern = spmv_slab_cg_kernel<kSlabThreads, kSlabUnroll>;
        LILAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kSlabCgSmemBytes + 64));
        done[A->device & 63] = 1;
    }
    return LILAC_OK;
}

// q = A p as slab partials (slab_P) and p.q as per-CTA sums (slab_pq).
inline lilac_status launch_slab_cg(lilac_csr_s* A, const double* p, const CgState* st,
                                   cudaStream_t stream) {
    LILAC_TRY(prepare_slab_cg(A));
    SlabView view{A->slab_cptr.as<int>(), A->slab_crow.as<int>(), A->slab_col.as<uint16_t>(),
                  A->slab_ctas.as<int4>(), A->slab_groups.as<int2>(), A->slab_gcnt.as<unsigned>(),
                  A->rows, A->ncols, A->slab_W, A->slab_S, A->slab_G};
    Scratch sc = A->scratch();
    sc.partials = A->slab_pq.as<double>();
    spmv_slab_cg_kernel<kSlabThreads, kSlabUnroll>
        <<<(unsigned)A->slab_grid, kSlabThreads, A->slab_cg_smem, stream>>>(
            view, A->slab_ranges.as<int4>(), A->slab_tsm, A->slab_val.as<double>(), p,
            A->slab_P.as<double>(), A->slab_T.as<double>(), st, sc);
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// SELL: the sliced ELL copy (lilac_sell.cu) with x gathered through L1/L2;
// split rows finish through the copy's own piece sums and counters.  Another
// value array (an FP32 copy) goes to STAGED, as does a handle without a copy.
constexpr int kSellThreads = 256;

// A two-phase epilogue with reductions runs as store + rows_reduce_kernel on
// a copy whose rows are sorted and many (sell_two_pass): reading x[row] and
// friends in sorted row order would scatter.
template <class Op>
bool sell_split_epilogue(const lilac_csr_s* A) {
    return Op::kTwoPhase && Op::NR > 0 && A->sell_two_pass;
}

template <int V, class Op>
lilac_status prepare_sell(lilac_csr_s* A) {
    int& bps = bps_slot<V + 256, Op, false>(A->device);
    if (bps == 0) {
        auto k1 = spmv_sell_kernel<kSellThreads, kSellUnroll, false, Op>;
        // no shared memory: the unified array goes to L1, which caches x
        LILAC_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        int b = occupancy_per_sm(k1, kSellThreads, 0);
        if constexpr (Op::kTwoPhase && Op::NR > 0) {
            auto k2 = spmv_sell_kernel<kSellThreads, kSellUnroll, true, Op>;
            LILAC_CUDA_TRY(cudaFuncSetAttribute(k2, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
            b = std::min(b, occupancy_per_sm(k2, kSellThreads, 0));
        }
        bps = b;
    }
    return prepare_staged_any<Op>(A);
}

template <int V, class Op>
lilac_status launch_sell(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                         const Op& op, cudaStream_t stream) {
    if (!A->sell_built || (const void*)val != A->val.p) return launch_staged_any<Op>(A, val, x, op, stream);
    LILAC_TRY(prepare_sell<V, Op>(A));
    const int bps = bps_slot<V + 256, Op, false>(A->device);
    constexpr int kWarps = kSellThreads / 32;
    int64_t grid = (int64_t)A->sm_count * bps;
    const int64_t need = ((int64_t)A->sell_nchunks + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    if (grid > kMaxCtas) grid = kMaxCtas;
    if (grid < 1) grid = 1;
    SellView view{A->sell_cptr.as<int>(), A->sell_crow.as<int>(), A->sell_col.as<int>(),
                  A->sell_splits.as<int4>(), A->sell_piece_split.as<int>(), A->sell_nchunks,
                  A->sell_nsplit};
    Scratch sc = A->scratch();
    sc.long_part = A->sell_part.as<double>();
    sc.long_red = A->sell_red.as<double>();
    sc.long_cnt = A->sell_cnt.as<unsigned>();
    if constexpr (Op::kTwoPhase && Op::NR > 0) {
        if (sell_split_epilogue<Op>(A)) {
            spmv_sell_kernel<kSellThreads, kSellUnroll, true, Op>
                <<<(unsigned)grid, kSellThreads, 0, stream>>>(view, A->sell_val.as<typename Op::ValT>(),
                                                              x, op, sc);
            LILAC_CUDA_TRY(cudaGetLastError());
            rows_reduce_kernel<kVecThreads, Op><<<vec_grid(A, A->rows), kVecThreads, 0, stream>>>(
                A->rows, op, A->scratch());
            LILAC_CUDA_TRY(cudaGetLastError());
            return LILAC_OK;
        }
    }
    {
        spmv_sell_kernel<kSellThreads, kSellUnroll, false, Op><<<(unsigned)grid, kSellThreads, 0, stream>>>(
            view, A->sell_val.as<typename Op::ValT>(), x, op, sc);
    }
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// HUB: the hub columns' x gathered, their pieces summed per slab from shared
// memory (hub_pieces_kernel), the cold part through the SELL kernel, which
// adds the slab partials (lilac_hub.cu builds the copies).  Another value
// array (an FP32 copy) goes to STAGED, as does a handle without the copies.
template <int V, class Op>
lilac_status prepare_hub(lilac_csr_s* A) {
    int& bps = bps_slot<V + 512, Op, true>(A->device);
    if (bps == 0) {
        auto kern = hub_pieces_kernel<kSlabThreads, kHubUnroll, Op>;
        LILAC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kSlabMaxBytes + 64));
        bps = 1;
    }
    // the cold part's SELL kernel (adding the slab sums): its own occupancy
    int& cps = bps_slot<V + 768, Op, false>(A->device);
    if (cps == 0) {
        auto k1 = spmv_sell_kernel<kSellThreads, kSellUnroll, false, Op, true>;
        LILAC_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        int b = occupancy_per_sm(k1, kSellThreads, 0);
        if constexpr (Op::kTwoPhase && Op::NR > 0) {
            auto k2 = spmv_sell_kernel<kSellThreads, kSellUnroll, true, Op, true>;
            LILAC_CUDA_TRY(cudaFuncSetAttribute(k2, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
            b = std::min(b, occupancy_per_sm(k2, kSellThreads, 0));
        }
        cps = b;
    }
    LILAC_TRY(prepare_sell<V, Op>(A));
    return prepare_staged_any<Op>(A);
}

template <class Op>
bool hub_split_epilogue(const lilac_csr_s* A) {
    return Op::kTwoPhase && Op::NR > 0 && A->hub_two_pass;
}

template <int V, class Op>
lilac_status launch_hub(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                        const Op& op, cudaStream_t stream) {
    if (!A->hub_built || (const void*)val != A->val.p) return launch_staged_any<Op>(A, val, x, op, stream);
    LILAC_TRY(prepare_hub<V, Op>(A));
    using VecT = typename Op::VecT;
    using AccT = typename Op::AccT;
    const int H = A->hub_H;
    VecT* xhot = A->hub_xhot.as<VecT>();
    hub_gather_kernel<VecT><<<(H + 255) / 256, 256, 0, stream>>>(H, A->hub_cols.as<int>(), x, xhot);
    LILAC_CUDA_TRY(cudaGetLastError());
    // rows: the stride of the slab partials P
    SlabView hv{A->hub_cptr.as<int>(), A->hub_crow.as<int>(), A->hub_col.as<uint16_t>(), nullptr,
                nullptr, nullptr, A->hub_pstride, H, A->hub_W, A->hub_S, 0};
    const size_t smem = (sizeof(VecT) * ((size_t)A->hub_W + 1) + 15) & ~size_t(15);
    const HubSplits hs{A->hub_splits.as<int4>(), A->hub_sub_split.as<int>(), A->hub_part.as<double>(),
                       A->hub_cnt.as<unsigned>()};
    hub_pieces_kernel<kSlabThreads, kHubUnroll, Op><<<(unsigned)A->hub_grid, kSlabThreads, smem, stream>>>(
        hv, A->hub_ranges.as<int4>(), A->hub_val.as<typename Op::ValT>(), xhot, H,
        A->hub_P.as<AccT>(), hs, op);
    LILAC_CUDA_TRY(cudaGetLastError());
    const int bps = bps_slot<V + 768, Op, false>(A->device);
    constexpr int kWarps = kSellThreads / 32;
    int64_t grid = (int64_t)A->sm_count * bps;
    const int64_t need = ((int64_t)A->hubc_nchunks + kWarps - 1) / kWarps;
    grid = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(grid, need), kMaxCtas));
    SellView cv{A->hubc_cptr.as<int>(), A->hubc_crow.as<int>(), A->hubc_col.as<int>(),
                A->hubc_splits.as<int4>(), A->hubc_piece_split.as<int>(), A->hubc_nchunks,
                A->hubc_nsplit, A->hub_P.p, A->hubc_mask.as<uint8_t>(), A->hub_pstride,
                32 * A->hubc_nchunks};
    Scratch sc = A->scratch();
    sc.long_part = A->hubc_part.as<double>();
    sc.long_red = A->hubc_red.as<double>();
    sc.long_cnt = A->hubc_cnt.as<unsigned>();
    if constexpr (Op::kTwoPhase && Op::NR > 0) {
        if (hub_split_epilogue<Op>(A)) {
            spmv_sell_kernel<kSellThreads, kSellUnroll, true, Op, true>
                <<<(unsigned)grid, kSellThreads, 0, stream>>>(cv, A->hubc_val.as<typename Op::ValT>(), x, op, sc);
            LILAC_CUDA_TRY(cudaGetLastError());
            rows_reduce_kernel<kVecThreads, Op><<<vec_grid(A, A->rows), kVecThreads, 0, stream>>>(
                A->rows, op, A->scratch());
            LILAC_CUDA_TRY(cudaGetLastError());
            return LILAC_OK;
        }
    }
    spmv_sell_kernel<kSellThreads, kSellUnroll, false, Op, true><<<(unsigned)grid, kSellThreads, 0, stream>>>(
        cv, A->hubc_val.as<typename Op::ValT>(), x, op, sc);
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

#define LILAC_DISPATCH_SPMV(FN_ROWS, FN_STAGED, FN_SLAB, FN_MERGE, FN_JDS, FN_SELL, FN_HUB, ...) \
    switch (A->variant) {                                                   \
        case LILAC_VARIANT_HUB: /* hub slabs + cold sliced ELL */           \
            return FN_HUB<1, Op>(__VA_ARGS__);                              \
        case LILAC_VARIANT_SELL: /* one lane per row piece */               \
            return FN_SELL<1, Op>(__VA_ARGS__);                             \
        case LILAC_VARIANT_MERGE: /* thread-sequential: no lanes per row */ \
            return FN_MERGE<1, Op>(__VA_ARGS__);                            \
        case LILAC_VARIANT_JDS: /* one thread per row */                    \
            return FN_JDS<1, Op>(__VA_ARGS__);                              \
        case LILAC_VARIANT_SLAB: /* one lane per row piece */               \
            return FN_SLAB<1, Op>(__VA_ARGS__);                             \
        case LILAC_VARIANT_SCALAR:                                          \
            return FN_ROWS<1, Op>(__VA_ARGS__);                             \
        case LILAC_VARIANT_VECTOR:                                          \
            switch (A->vwidth) {                                            \
                case 2: return FN_ROWS<2, Op>(__VA_ARGS__);                 \
                case 4: return FN_ROWS<4, Op>(__VA_ARGS__);                 \
                case 8: return FN_ROWS<8, Op>(__VA_ARGS__);                 \
                case 16: return FN_ROWS<16, Op>(__VA_ARGS__);               \
                default: return FN_ROWS<32, Op>(__VA_ARGS__);               \
            }                                                               \
        case LILAC_VARIANT_STAGED:                                          \
        default:                                                            \
            switch (A->vwidth) {                                            \
                case 1: return FN_STAGED<1, Op>(__VA_ARGS__);               \
                case 2: return FN_STAGED<2, Op>(__VA_ARGS__);               \
                case 4: return FN_STAGED<4, Op>(__VA_ARGS__);               \
                case 8: return FN_STAGED<8, Op>(__VA_ARGS__);               \
                case 16: return FN_STAGED<16, Op>(__VA_ARGS__);             \
                default: return FN_STAGED<32, Op>(__VA_ARGS__);             \
            }                                                               \
    }

// SLAB launches fall back to STAGED in some cases, so prepare both.
template <int V, class Op>
lilac_status prepare_slab_and_staged(lilac_csr_s* A) {
    LILAC_TRY(prepare_slab<V, Op>(A));
    return prepare_staged_any<Op>(A);
}

// Kernel launches one SpMV with epilogue Op of the handle's variant makes
// with value array `val` (SELL with a split epilogue: the SpMV and the
// row-order reduction).
template <class Op>
int spmv_launch_count(const lilac_csr_s* A, const void* val) {
    if (val != A->val.p) return 1;
    if (A->variant == LILAC_VARIANT_SELL && A->sell_built && sell_split_epilogue<Op>(A)) return 2;
    if (A->variant == LILAC_VARIANT_HUB && A->hub_built) return hub_split_epilogue<Op>(A) ? 4 : 3;
    return 1;
}

template <class Op>
lilac_status prepare_spmv(lilac_csr_s* A) {
    LILAC_DISPATCH_SPMV(prepare_rows, prepare_staged, prepare_slab_and_staged, prepare_merge,
                        prepare_jds, prepare_sell, prepare_hub, A)
}

template <class Op>
lilac_status launch_spmv(lilac_csr_s* A, const typename Op::ValT* val, const typename Op::VecT* x,
                         const Op& op, cudaStream_t stream) {
    LILAC_DISPATCH_SPMV(launch_rows, launch_staged, launch_slab, launch_merge, launch_jds,
                        launch_sell, launch_hub, A, val, x, op, stream)
}

// Replay `body` (which enqueues work on the stream it is given) as a CUDA
// graph captured once per key and cached in the handle, or run it directly.
// Everything `body` launches must have been prepared (prepare_spmv) first.
template <class F>
lilac_status run_maybe_graph(lilac_csr_s* A, const GraphKey& key, bool use_graph,
                             cudaStream_t stream, F&& body) {
    if (!use_graph) return body(stream);
    auto it = A->graphs.find(key);
    if (it == A->graphs.end()) {
        if (A->graphs.size() >= 64) {
            for (auto& kv : A->graphs) cudaGraphExecDestroy(kv.second);
            A->graphs.clear();
        }
        if (!A->capture_stream)
            LILAC_CUDA_TRY(cudaStreamCreateWithFlags(&A->capture_stream, cudaStreamNonBlocking));
        LILAC_CUDA_TRY(cudaStreamBeginCapture(A->capture_stream, cudaStreamCaptureModeThreadLocal));
        lilac_status st = body(A->capture_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(A->capture_stream, &g);
        if (st != LILAC_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) {
            set_last_error(std::string("stream capture: ") + cudaGetErrorString(e));
            return LILAC_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            set_last_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            return LILAC_ERR_CUDA;
        }
        it = A->graphs.emplace(key, ex).first;
    }
    LILAC_CUDA_TRY(cudaGraphLaunch(it->second, stream));
    return LILAC_OK;
}

}  // namespace lilac
