// Regrouped copy of a matrix for the SLAB kernel (row blocks x column
// slabs), built once per handle on first use and kept with it, like the
// other invariants cached at create.
//
// Rows are cut into blocks of kSlabBlockRows; columns into slabs of
// kSlabWidth.  Unit (b, s) = the nonzeros of block b whose columns lie in
// slab s.  Storage is slab-major (slab, then block, then row; CSR order
// inside a row) with local columns c - s*W and one row-pointer array per
// unit (block rows + 1 absolute offsets).  Tiles of at most kSlabTileNnz
// nonzeros and kSlabTileRows rows never cross a unit.  Non-empty units are
// dealt, in storage order, to CTAs in contiguous runs of about equal
// nonzero count; a run never touches more than two slabs (the kernel holds
// two slabs of x), so runs are split where needed.
#include <algorithm>
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace lilac {

bool slab_worthwhile(const lilac_csr_s* A) {
    if (A->nnz == 0 || A->ncols == 0) return false;
    const int64_t S = (A->ncols + kSlabWidth - 1) / kSlabWidth;
    // each CTA's share of the nonzeros should cover whole slabs' worth of
    // gathers: at least ~16 nonzeros per column on average, few slabs
    return (double)A->nnz / (double)A->ncols >= 16.0 && S <= 64;
}

template <class T>
static lilac_status build_slab(lilac_csr A, cudaStream_t s) {
    const int n = A->rows;
    const int64_t nnz = A->nnz;
    const int W = kSlabWidth, RB = kSlabBlockRows;
    const int S = A->ncols > 0 ? (A->ncols + W - 1) / W : 0;
    const int NB = (n + RB - 1) / RB;
    std::vector<int32_t> col((size_t)nnz);
    std::vector<T> val((size_t)nnz);
    if (nnz > 0) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(col.data(), A->col_ind.p, sizeof(int32_t) * (size_t)nnz,
                                       cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaMemcpyAsync(val.data(), A->val.p, sizeof(T) * (size_t)nnz,
                                       cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    const auto& rp = A->h_row_ptr;
    // entries per (row, slab)
    std::vector<int32_t> rs_cnt((size_t)n * std::max(1, S), 0);
    for (int r = 0; r < n; ++r)
        for (int j = rp[r]; j < rp[r + 1]; ++j) rs_cnt[(size_t)r * S + col[j] / W]++;
    // units in storage order, their row pointers and tiles
    std::vector<SlabBlock> blocks((size_t)NB);
    for (int b = 0; b < NB; ++b) blocks[b] = {b * RB, std::min(RB, n - b * RB), 0, 0};
    struct Unit { int b, s; int64_t k0, k1; int tile_begin, tile_end; int64_t lrp_base; };
    std::vector<Unit> units;
    std::vector<int32_t> lrp;
    std::vector<int64_t> next((size_t)n * std::max(1, S));
    int64_t pos = 0;
    for (int sl = 0; sl < S; ++sl)
        for (int b = 0; b < NB; ++b) {
            const SlabBlock& B = blocks[b];
            const int64_t base = (int64_t)lrp.size();
            const int64_t k0 = pos;
            for (int r = B.r0; r < B.r0 + B.nrows; ++r) {
                lrp.push_back((int32_t)pos);
                next[(size_t)r * S + sl] = pos;
                pos += rs_cnt[(size_t)r * S + sl];
            }
            lrp.push_back((int32_t)pos);
            if (pos > k0) {
                units.push_back({b, sl, k0, pos, 0, 0, base});
                blocks[b].need++;
            }
        }
    std::vector<T> sval((size_t)((nnz + 11) & ~3ll));
    std::vector<int32_t> scol((size_t)((nnz + 11) & ~3ll), 0);
    std::vector<int32_t> perm((size_t)std::max<int64_t>(1, nnz));
    for (int r = 0; r < n; ++r)
        for (int j = rp[r]; j < rp[r + 1]; ++j) {
            const int sl = col[j] / W;
            const int64_t q = next[(size_t)r * S + sl]++;
            sval[(size_t)q] = val[(size_t)j];
            scol[(size_t)q] = col[j] - sl * W;
            perm[(size_t)q] = j;
        }
    // tiles per unit
    std::vector<SlabTile> tiles;
    for (Unit& u : units) {
        const int nr = blocks[u.b].nrows;
        const int32_t* Lp = &lrp[(size_t)u.lrp_base];
        u.tile_begin = (int)tiles.size();
        int64_t k = u.k0;
        int rl = 0;
        while (k < u.k1) {
            while (Lp[rl + 1] <= k) ++rl;  // first row that ends after k
            int64_t k1 = std::min<int64_t>(u.k1, k + kSlabTileNnz);
            int re = rl;
            while (re < nr && Lp[re] < k1) ++re;  // rows [rl, re) start before k1
            if (re - rl > kSlabTileRows) {
                re = rl + kSlabTileRows;
                k1 = Lp[re];
            }
            tiles.push_back({(int)k, (int)k1, (int)(u.lrp_base + rl), rl, re - rl, u.s, u.b, 0});
            k = k1;
        }
        tiles.back().last = 1;
        u.tile_end = (int)tiles.size();
    }
    // CTA runs: contiguous units, about nnz / sm_count each, at most two slabs
    std::vector<int2> cta_tiles, cta_slabs;
    const int64_t target = std::max<int64_t>(1, (nnz + A->sm_count - 1) / A->sm_count);
    size_t u = 0;
    while (u < units.size()) {
        const size_t u0 = u;
        int64_t acc = 0;
        int s_a = units[u].s, s_b = -1;
        while (u < units.size() && (acc < target || u == u0)) {
            const int su = units[u].s;
            if (su != s_a) {
                if (s_b < 0)
                    s_b = su;
                else if (su != s_b)
                    break;
            }
            acc += units[u].k1 - units[u].k0;
            ++u;
        }
        cta_tiles.push_back(make_int2(units[u0].tile_begin, units[u - 1].tile_end));
        cta_slabs.push_back(make_int2(s_a, s_b));
    }
    if (cta_tiles.empty()) {  // no nonzero at all: one CTA writes the zero rows
        cta_tiles.push_back(make_int2(0, 0));
        cta_slabs.push_back(make_int2(-1, -1));
    }
    lrp.resize(lrp.size() + 8, lrp.empty() ? 0 : lrp.back());  // padding for rounded-up copies
    LILAC_TRY(A->ws_alloc(A->slab_val, sizeof(T) * sval.size()));
    LILAC_TRY(A->ws_alloc(A->slab_col, sizeof(int32_t) * scol.size()));
    LILAC_TRY(A->ws_alloc(A->slab_lrp, sizeof(int32_t) * lrp.size()));
    LILAC_TRY(A->ws_alloc(A->slab_blocks, sizeof(SlabBlock) * std::max<size_t>(1, blocks.size())));
    LILAC_TRY(A->ws_alloc(A->slab_tiles, sizeof(SlabTile) * std::max<size_t>(1, tiles.size())));
    LILAC_TRY(A->ws_alloc(A->slab_perm, sizeof(int32_t) * perm.size()));
    LILAC_TRY(A->ws_alloc(A->slab_cta_tiles, sizeof(int2) * cta_tiles.size()));
    LILAC_TRY(A->ws_alloc(A->slab_cta_slabs, sizeof(int2) * cta_slabs.size()));
    LILAC_TRY(A->ws_alloc(A->slab_P, sizeof(double) * (size_t)std::max(1, S) * (size_t)std::max(1, n)));
    LILAC_TRY(A->ws_alloc(A->slab_cnt, sizeof(unsigned) * std::max<size_t>(1, blocks.size())));
    LILAC_TRY(A->ws_alloc(A->slab_block_red, sizeof(double) * kMaxRed * std::max<size_t>(1, blocks.size())));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_P.p, 0, A->slab_P.bytes, s));  // empty units stay 0
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_cnt.p, 0, A->slab_cnt.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_block_red.p, 0, A->slab_block_red.bytes, s));
    auto up = [&](lilac::DevBuf& d, const void* h, size_t bytes) -> lilac_status {
        if (bytes) LILAC_CUDA_TRY(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, s));
        return LILAC_OK;
    };
    LILAC_TRY(up(A->slab_val, sval.data(), sizeof(T) * sval.size()));
    LILAC_TRY(up(A->slab_col, scol.data(), sizeof(int32_t) * scol.size()));
    LILAC_TRY(up(A->slab_lrp, lrp.data(), sizeof(int32_t) * lrp.size()));
    LILAC_TRY(up(A->slab_blocks, blocks.data(), sizeof(SlabBlock) * blocks.size()));
    LILAC_TRY(up(A->slab_tiles, tiles.data(), sizeof(SlabTile) * tiles.size()));
    LILAC_TRY(up(A->slab_perm, perm.data(), sizeof(int32_t) * perm.size()));
    LILAC_TRY(up(A->slab_cta_tiles, cta_tiles.data(), sizeof(int2) * cta_tiles.size()));
    LILAC_TRY(up(A->slab_cta_slabs, cta_slabs.data(), sizeof(int2) * cta_slabs.size()));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->slab_nblocks = (int)blocks.size();
    A->slab_ntiles = (int)tiles.size();
    A->slab_nslabs = S;
    A->slab_grid = (int)cta_tiles.size();
    A->slab_built = true;
    return LILAC_OK;
}

template <class T>
__global__ void slab_regather_kernel(int64_t nnz, const int* __restrict__ perm,
                                     const T* __restrict__ val, T* __restrict__ sval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        sval[q] = val[perm[q]];
}

// After new values were uploaded: rebuild the regrouped values on the device.
lilac_status slab_refresh_values(lilac_csr A, cudaStream_t s) {
    if (!A->slab_built || A->nnz == 0) return LILAC_OK;
    if (A->dtype == LILAC_F64)
        slab_regather_kernel<double><<<A->sm_count * 8, 256, 0, s>>>(
            A->nnz, A->slab_perm.as<int>(), A->val.as<double>(), A->slab_val.as<double>());
    else
        slab_regather_kernel<float><<<A->sm_count * 8, 256, 0, s>>>(
            A->nnz, A->slab_perm.as<int>(), A->val.as<float>(), A->slab_val.as<float>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

lilac_status ensure_slab(lilac_csr A, cudaStream_t s) {
    if (A->slab_built) return LILAC_OK;
    const int64_t S = A->ncols > 0 ? (A->ncols + kSlabWidth - 1) / kSlabWidth : 0;
    // per (row, slab) counters and row pointers: (slabs) x (rows + blocks) entries
    if (S > 256 || S * (2 * (int64_t)A->rows + 2) >= (int64_t(1) << 31) - 64) {
        set_last_error("matrix has too many column slabs for the SLAB layout");
        return LILAC_ERR_UNSUPPORTED;
    }
    return A->dtype == LILAC_F64 ? build_slab<double>(A, s) : build_slab<float>(A, s);
}

}  // namespace lilac
