// Regrouped copy of a matrix for the SLAB kernel (row blocks x column
// slabs), built once per handle on first use and kept with it, like the
// other invariants cached at create.
//
// Row blocks: consecutive rows, about nnz / (number of SMs) nonzeros each and
// at most kSlabBlockRows rows.  Within block b the nonzeros are stored slab
// by slab (slab s = columns [s*W, (s+1)*W)), row by row inside a slab, in
// their CSR order inside a row, with local column c - s*W.  For each (b, s)
// a row-pointer array of (rows in b) + 1 absolute offsets is stored.  Tiles
// of at most kSlabTileNnz nonzeros and kSlabTileRows rows never cross a slab.
#include <algorithm>
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace lilac {

bool slab_worthwhile(const lilac_csr_s* A) {
    if (A->nnz == 0 || A->ncols == 0) return false;
    const double vsz = A->dtype == LILAC_F64 ? 8.0 : 4.0;
    const double x_loads = (double)A->sm_count * (double)A->ncols * vsz;  // x read once per CTA
    const double matrix = (double)A->nnz * (vsz + 4.0);
    return x_loads <= 4.0 * matrix;
}

template <class T>
static lilac_status build_slab(lilac_csr A, cudaStream_t s) {
    const int n = A->rows;
    const int64_t nnz = A->nnz;
    const int W = kSlabWidth;
    const int S = A->ncols > 0 ? (A->ncols + W - 1) / W : 0;
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
    // row blocks
    const int64_t target = std::max<int64_t>(1, (nnz + A->sm_count - 1) / A->sm_count);
    std::vector<SlabBlock> blocks;
    for (int r = 0; r < n;) {
        const int r0 = r;
        int64_t cnt = 0;
        while (r < n && r - r0 < kSlabBlockRows && (cnt < target || r == r0)) {
            cnt += rp[r + 1] - rp[r];
            ++r;
        }
        blocks.push_back({r0, r - r0, 0, 0});
    }
    std::vector<T> sval((size_t)((nnz + 11) & ~3ll));
    std::vector<int32_t> scol((size_t)((nnz + 11) & ~3ll), 0);
    std::vector<int32_t> perm((size_t)std::max<int64_t>(1, nnz));  // regrouped position -> CSR position
    std::vector<int32_t> lrp;
    std::vector<SlabTile> tiles;
    std::vector<int64_t> seg_cnt((size_t)std::max(1, S));
    int64_t pos = 0;  // running position in the regrouped arrays
    for (SlabBlock& B : blocks) {
        const int r0 = B.r0, nr = B.nrows;
        // entries of each (row, slab) of the block: counts, then placement
        std::fill(seg_cnt.begin(), seg_cnt.end(), 0);
        for (int r = r0; r < r0 + nr; ++r)
            for (int j = rp[r]; j < rp[r + 1]; ++j) seg_cnt[col[j] / W]++;
        std::vector<int64_t> seg_start((size_t)std::max(1, S));
        int64_t acc = pos;
        for (int sl = 0; sl < S; ++sl) {
            seg_start[sl] = acc;
            acc += seg_cnt[sl];
        }
        // row pointers of each (block, slab): lrp_base[sl] .. + nr
        std::vector<int64_t> lrp_base((size_t)std::max(1, S));
        for (int sl = 0; sl < S; ++sl) {
            lrp_base[sl] = (int64_t)lrp.size();
            lrp.resize(lrp.size() + (size_t)nr + 1);
        }
        std::vector<int64_t> fill(seg_start.begin(), seg_start.end());
        for (int r = r0; r < r0 + nr; ++r) {
            for (int sl = 0; sl < S; ++sl) lrp[(size_t)(lrp_base[sl] + (r - r0))] = (int32_t)fill[sl];
            for (int j = rp[r]; j < rp[r + 1]; ++j) {
                const int sl = col[j] / W;
                const int64_t q = fill[sl]++;
                sval[(size_t)q] = val[(size_t)j];
                scol[(size_t)q] = col[j] - sl * W;
                perm[(size_t)q] = j;
            }
        }
        for (int sl = 0; sl < S; ++sl) lrp[(size_t)(lrp_base[sl] + nr)] = (int32_t)fill[sl];
        // tiles of each non-empty slab segment
        B.tile_begin = (int)tiles.size();
        std::vector<int> used;
        for (int sl = 0; sl < S; ++sl)
            if (seg_cnt[sl] > 0) used.push_back(sl);
        for (size_t u = 0; u < used.size(); ++u) {
            const int sl = used[u];
            const int nxt = u + 1 < used.size() ? used[u + 1] : -1;
            const int32_t* L = &lrp[(size_t)lrp_base[sl]];
            const int64_t kend = seg_start[sl] + seg_cnt[sl];
            int64_t k = seg_start[sl];
            int rl = 0;
            bool first = true;
            while (k < kend) {
                while (L[rl + 1] <= k) ++rl;  // first row that ends after k
                int64_t k1 = std::min<int64_t>(kend, k + kSlabTileNnz);
                int re = rl;
                while (re < nr && L[re] < k1) ++re;  // rows [rl, re) start before k1
                if (re - rl > kSlabTileRows) {
                    re = rl + kSlabTileRows;
                    k1 = L[re];
                }
                SlabTile t;
                t.k0 = (int)k;
                t.k1 = (int)k1;
                t.lrp_idx = (int)(lrp_base[sl] + rl);
                t.rl0 = rl;
                t.nrows = re - rl;
                t.slab = sl;
                t.next_slab = first ? nxt : -1;
                t.first = first ? 1 : 0;
                tiles.push_back(t);
                first = false;
                k = k1;
            }
        }
        B.tile_end = (int)tiles.size();
        pos = acc;
    }
    lrp.resize(lrp.size() + 8, lrp.empty() ? 0 : lrp.back());  // padding for rounded-up copies
    LILAC_TRY(A->ws_alloc(A->slab_val, sizeof(T) * sval.size()));
    LILAC_TRY(A->ws_alloc(A->slab_col, sizeof(int32_t) * scol.size()));
    LILAC_TRY(A->ws_alloc(A->slab_lrp, sizeof(int32_t) * lrp.size()));
    LILAC_TRY(A->ws_alloc(A->slab_blocks, sizeof(SlabBlock) * std::max<size_t>(1, blocks.size())));
    LILAC_TRY(A->ws_alloc(A->slab_tiles, sizeof(SlabTile) * std::max<size_t>(1, tiles.size())));
    LILAC_TRY(A->ws_alloc(A->slab_perm, sizeof(int32_t) * perm.size()));
    LILAC_CUDA_TRY(cudaMemcpyAsync(A->slab_perm.p, perm.data(), sizeof(int32_t) * perm.size(),
                                   cudaMemcpyHostToDevice, s));
    LILAC_CUDA_TRY(cudaMemcpyAsync(A->slab_val.p, sval.data(), sizeof(T) * sval.size(),
                                   cudaMemcpyHostToDevice, s));
    LILAC_CUDA_TRY(cudaMemcpyAsync(A->slab_col.p, scol.data(), sizeof(int32_t) * scol.size(),
                                   cudaMemcpyHostToDevice, s));
    LILAC_CUDA_TRY(cudaMemcpyAsync(A->slab_lrp.p, lrp.data(), sizeof(int32_t) * lrp.size(),
                                   cudaMemcpyHostToDevice, s));
    if (!blocks.empty())
        LILAC_CUDA_TRY(cudaMemcpyAsync(A->slab_blocks.p, blocks.data(),
                                       sizeof(SlabBlock) * blocks.size(), cudaMemcpyHostToDevice, s));
    if (!tiles.empty())
        LILAC_CUDA_TRY(cudaMemcpyAsync(A->slab_tiles.p, tiles.data(), sizeof(SlabTile) * tiles.size(),
                                       cudaMemcpyHostToDevice, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->slab_nblocks = (int)blocks.size();
    A->slab_ntiles = (int)tiles.size();
    A->slab_nslabs = S;
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
    // row pointers: (slabs) x (rows + blocks) int32 entries
    const int64_t S = A->ncols > 0 ? (A->ncols + kSlabWidth - 1) / kSlabWidth : 0;
    if (S * (2 * (int64_t)A->rows + 2) >= (int64_t(1) << 31) - 64) {
        set_last_error("matrix too large for the SLAB layout's 32-bit row pointers");
        return LILAC_ERR_UNSUPPORTED;
    }
    return A->dtype == LILAC_F64 ? build_slab<double>(A, s) : build_slab<float>(A, s);
}

}  // namespace lilac
