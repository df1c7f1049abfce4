// Regrouped copy of a matrix for the SLAB kernels, built once per handle on
// first use (or for the tuner's trial) and kept with it, like the other
// invariants cached at create.
//
// The columns are cut into S slabs of W columns, W * 8 bytes at most
// kSlabMaxBytes, S as small as that allows.  Sub-matrix A_s holds, for every
// row, the nonzeros whose column lies in [s W, (s+1) W), in CSR order, with
// 16-bit local columns c - s W; the sub-matrices are stored one after the
// other, each with its own row pointers (absolute offsets).  The rows of each
// A_s are cut into G = SMs / S runs of about equal nonzero count, one per
// CTA.  A permutation (regrouped position -> CSR position) re-gathers the
// values after lilac_csr_update_values.
#include <algorithm>
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace lilac {

namespace {

int slab_count(const lilac_csr_s* A, int* W) {
    const int64_t per = kSlabMaxBytes / 8;
    const int64_t S = A->ncols > 0 ? (A->ncols + per - 1) / per : 0;
    int64_t w = S > 0 ? (A->ncols + S - 1) / S : 0;
    w = (w + 7) & ~int64_t(7);
    *W = (int)w;
    return (int)S;
}

}  // namespace

// Worth building when x is too large for L1 yet a handful of slabs holds it,
// each CTA's share of the nonzeros is large, and rows are long enough per
// slab to amortise the per-row work.
bool slab_worthwhile(const lilac_csr_s* A) {
    if (A->nnz == 0 || A->rows == 0 || A->ncols == 0) return false;
    int W = 0;
    const int S = slab_count(A, &W);
    return (int64_t)A->ncols * 8 > (128 << 10) && S <= 8 && S <= A->sm_count &&
           A->mean_row_len >= 8.0 * S && A->nnz >= (int64_t)A->sm_count * 4096;
}

template <class T>
__global__ void slab_regather_kernel(int64_t nnz, const int* __restrict__ perm,
                                     const T* __restrict__ val, T* __restrict__ sval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * blockDim.x)
        sval[q] = val[perm[q]];
}

template <class T>
static lilac_status regather(lilac_csr A, cudaStream_t s) {
    if (A->nnz == 0) return LILAC_OK;
    slab_regather_kernel<T><<<A->sm_count * 8, 256, 0, s>>>(A->nnz, A->slab_perm.as<int>(),
                                                             A->val.as<T>(), A->slab_val.as<T>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

static lilac_status build_slab(lilac_csr A, cudaStream_t s) {
    const int n = A->rows;
    const int64_t nnz = A->nnz;
    int W = 0;
    const int S = slab_count(A, &W);
    const auto& rp = A->h_row_ptr;
    std::vector<int32_t> col((size_t)nnz);
    LILAC_CUDA_TRY(cudaMemcpyAsync(col.data(), A->col_ind.p, sizeof(int32_t) * (size_t)nnz,
                                   cudaMemcpyDeviceToHost, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    // per-slab row pointers, rows padded to a multiple of 4 ints (16 bytes)
    const int stride = ((n + 1) + 3) & ~3;
    std::vector<int32_t> srp((size_t)S * (size_t)stride, 0);
    {
        std::vector<int32_t> cnt((size_t)S * (size_t)std::max(1, n), 0);
        for (int r = 0; r < n; ++r)
            for (int k = rp[r]; k < rp[r + 1]; ++k) cnt[(size_t)(col[(size_t)k] / W) * n + r]++;
        int64_t base = 0;
        for (int sl = 0; sl < S; ++sl) {
            int32_t* p = srp.data() + (size_t)sl * stride;
            p[0] = (int32_t)base;
            for (int r = 0; r < n; ++r) {
                p[r + 1] = p[r] + cnt[(size_t)sl * n + r];
            }
            for (int r = n + 1; r < stride; ++r) p[r] = p[n];
            base = p[n];
        }
    }
    // regrouped local columns and the permutation
    std::vector<int32_t> perm((size_t)nnz);
    std::vector<uint16_t> c16((size_t)nnz);
    {
        std::vector<int32_t> pos((size_t)S);
        for (int r = 0; r < n; ++r) {
            for (int sl = 0; sl < S; ++sl) pos[(size_t)sl] = srp[(size_t)sl * stride + r];
            for (int k = rp[r]; k < rp[r + 1]; ++k) {
                const int c = col[(size_t)k];
                const int sl = c / W;
                const int32_t q = pos[(size_t)sl]++;
                perm[(size_t)q] = k;
                c16[(size_t)q] = (uint16_t)(c - sl * W);
            }
        }
    }
    // runs of rows of about equal nonzero count per slab, one per CTA
    const int G = std::max(1, A->sm_count / std::max(1, S));
    std::vector<int4> ctas;
    for (int sl = 0; sl < S; ++sl) {
        const int32_t* p = srp.data() + (size_t)sl * stride;
        const int64_t k0 = p[0], tot = (int64_t)p[n] - k0;
        int r = 0;
        for (int g = 0; g < G && r < n; ++g) {
            const int r0 = r;
            const int64_t target = k0 + tot * (g + 1) / G;
            if (g == G - 1)
                r = n;
            else
                while (r < n && p[r + 1] <= target) ++r;
            if (r > r0) ctas.push_back(make_int4(sl, r0, r, 0));
        }
        if (r < n) ctas.push_back(make_int4(sl, r, n, 0));
    }
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    const size_t npad = (size_t)nnz + 16;
    LILAC_TRY(A->ws_alloc(A->slab_rp, sizeof(int32_t) * srp.size()));
    LILAC_TRY(A->ws_alloc(A->slab_col, sizeof(uint16_t) * npad));
    LILAC_TRY(A->ws_alloc(A->slab_val, vsz * npad));
    LILAC_TRY(A->ws_alloc(A->slab_perm, sizeof(int32_t) * (size_t)std::max<int64_t>(1, nnz)));
    LILAC_TRY(A->ws_alloc(A->slab_ctas, sizeof(int4) * std::max<size_t>(1, ctas.size())));
    LILAC_TRY(A->ws_alloc(A->slab_P, sizeof(double) * (size_t)S * (size_t)std::max(1, n)));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_col.p, 0, A->slab_col.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_val.p, 0, A->slab_val.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_P.p, 0, A->slab_P.bytes, s));
    auto up = [&](lilac::DevBuf& d, const void* h, size_t bytes) -> lilac_status {
        if (bytes) LILAC_CUDA_TRY(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, s));
        return LILAC_OK;
    };
    LILAC_TRY(up(A->slab_rp, srp.data(), sizeof(int32_t) * srp.size()));
    LILAC_TRY(up(A->slab_col, c16.data(), sizeof(uint16_t) * c16.size()));
    LILAC_TRY(up(A->slab_perm, perm.data(), sizeof(int32_t) * perm.size()));
    LILAC_TRY(up(A->slab_ctas, ctas.data(), sizeof(int4) * ctas.size()));
    LILAC_TRY(A->dtype == LILAC_F64 ? regather<double>(A, s) : regather<float>(A, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->slab_S = S;
    A->slab_W = W;
    A->slab_grid = (int)ctas.size();
    A->slab_rp_stride = stride;
    A->slab_built = !ctas.empty();
    return LILAC_OK;
}

// After new values were uploaded: rebuild the regrouped values on the device.
lilac_status slab_refresh_values(lilac_csr A, cudaStream_t s) {
    if (!A->slab_built) return LILAC_OK;
    return A->dtype == LILAC_F64 ? regather<double>(A, s) : regather<float>(A, s);
}

void slab_release(lilac_csr A) {
    lilac::DevBuf* b[] = {&A->slab_rp, &A->slab_col, &A->slab_val, &A->slab_perm, &A->slab_ctas,
                          &A->slab_P};
    for (auto* d : b) d->release();
    A->slab_S = A->slab_W = A->slab_grid = A->slab_rp_stride = 0;
    A->slab_built = false;
}

lilac_status ensure_slab(lilac_csr A, cudaStream_t s) {
    if (A->slab_built) return LILAC_OK;
    int W = 0;
    const int S = slab_count(A, &W);
    if (A->nnz == 0 || S == 0) return LILAC_OK;  // nothing to regroup: STAGED runs
    // too many slabs for the layout: not built, STAGED runs
    if (S > 64 || (int64_t)S * ((int64_t)A->rows + 4) >= (int64_t(1) << 31) - 64) return LILAC_OK;
    return build_slab(A, s);
}

}  // namespace lilac
