// Jagged diagonal storage of a handle's matrix (the JDS format of Section
// 3.2), built once on first use and kept with the handle like the other
// invariants cached at create.
//
// Slots are the rows sorted by length, longest first (a stable counting
// sort: rows of equal length keep their order), so perm[r] = slot of row r.
// Jagged diagonal d holds the d-th nonzero of every slot whose row is longer
// than d, in slot order, at [jd_ptr[d], jd_ptr[d+1]).  The permutation and
// the diagonal offsets come from the host copy of row_ptr; columns and
// values are scattered into place on the device, one warp per row.
#include <algorithm>
#include <vector>

#include "launch.cuh"

namespace lilac {

template <class T>
__global__ void jds_scatter_kernel(int rows, const int* __restrict__ row_ptr,
                                   const int* __restrict__ row_slot, const int* __restrict__ jd_ptr,
                                   const int* __restrict__ col, const T* __restrict__ val,
                                   int* __restrict__ jcol, T* __restrict__ jval) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int r = warp; r < rows; r += nwarps) {
        const int k0 = row_ptr[r], k1 = row_ptr[r + 1], sl = row_slot[r];
        for (int d = lane; d < k1 - k0; d += 32) {
            const int k = jd_ptr[d] + sl;
            if (jcol) jcol[k] = col[k0 + d];
            jval[k] = val[k0 + d];
        }
    }
}

template <class T>
static lilac_status jds_scatter(lilac_csr A, bool with_cols, cudaStream_t s) {
    if (A->nnz == 0) return LILAC_OK;
    jds_scatter_kernel<T><<<A->sm_count * 8, 256, 0, s>>>(
        A->rows, A->row_ptr.as<int>(), A->jds_row_slot.as<int>(), A->jds_ptr.as<int>(),
        A->col_ind.as<int>(), A->val.as<T>(), with_cols ? A->jds_col.as<int>() : nullptr,
        A->jds_val.as<T>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

static lilac_status build_jds(lilac_csr A, cudaStream_t s) {
    const int n = A->rows;
    const auto& rp = A->h_row_ptr;
    const int maxlen = A->max_row_len;
    // stable counting sort by length, longest first
    std::vector<int32_t> start((size_t)maxlen + 2, 0);
    for (int r = 0; r < n; ++r) start[(size_t)(maxlen - (rp[r + 1] - rp[r]))]++;
    int32_t acc = 0;
    for (auto& c : start) {
        const int32_t t = c;
        c = acc;
        acc += t;
    }
    std::vector<int32_t> slot_row((size_t)n), row_slot((size_t)n), len((size_t)n);
    for (int r = 0; r < n; ++r) {
        const int L = rp[r + 1] - rp[r];
        const int32_t sl = start[(size_t)(maxlen - L)]++;
        row_slot[(size_t)r] = sl;
        slot_row[(size_t)sl] = r;
        len[(size_t)sl] = L;
    }
    // jd_ptr[d + 1] - jd_ptr[d] = slots longer than d (slots are sorted)
    std::vector<int32_t> jd_ptr((size_t)maxlen + 1, 0);
    {
        int32_t cnt = n;  // slots with len > d, d rising
        int sl = n - 1;
        for (int d = 0; d < maxlen; ++d) {
            while (sl >= 0 && len[(size_t)sl] <= d) {
                --sl;
                --cnt;
            }
            jd_ptr[(size_t)d + 1] = jd_ptr[(size_t)d] + cnt;
        }
    }
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    LILAC_TRY(A->ws_alloc(A->jds_slot_row, sizeof(int32_t) * std::max<size_t>(1, (size_t)n)));
    LILAC_TRY(A->ws_alloc(A->jds_row_slot, sizeof(int32_t) * std::max<size_t>(1, (size_t)n)));
    LILAC_TRY(A->ws_alloc(A->jds_len, sizeof(int32_t) * std::max<size_t>(1, (size_t)n)));
    LILAC_TRY(A->ws_alloc(A->jds_ptr, sizeof(int32_t) * jd_ptr.size()));
    LILAC_TRY(A->ws_alloc(A->jds_col, sizeof(int32_t) * std::max<int64_t>(1, A->nnz)));
    LILAC_TRY(A->ws_alloc(A->jds_val, vsz * (size_t)std::max<int64_t>(1, A->nnz)));
    auto up = [&](lilac::DevBuf& d, const std::vector<int32_t>& h) -> lilac_status {
        if (!h.empty())
            LILAC_CUDA_TRY(cudaMemcpyAsync(d.p, h.data(), sizeof(int32_t) * h.size(),
                                           cudaMemcpyHostToDevice, s));
        return LILAC_OK;
    };
    LILAC_TRY(up(A->jds_slot_row, slot_row));
    LILAC_TRY(up(A->jds_row_slot, row_slot));
    LILAC_TRY(up(A->jds_len, len));
    LILAC_TRY(up(A->jds_ptr, jd_ptr));
    LILAC_TRY(A->dtype == LILAC_F64 ? jds_scatter<double>(A, true, s) : jds_scatter<float>(A, true, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->jds_njd = maxlen;
    A->jds_built = true;
    return LILAC_OK;
}

lilac_status ensure_jds(lilac_csr A, cudaStream_t s) {
    if (A->jds_built) return LILAC_OK;
    return build_jds(A, s);
}

// After new values were uploaded: scatter them into JDS order again.
lilac_status jds_refresh_values(lilac_csr A, cudaStream_t s) {
    if (!A->jds_built) return LILAC_OK;
    return A->dtype == LILAC_F64 ? jds_scatter<double>(A, false, s) : jds_scatter<float>(A, false, s);
}

void jds_release(lilac_csr A) {
    A->jds_slot_row.release();
    A->jds_row_slot.release();
    A->jds_len.release();
    A->jds_ptr.release();
    A->jds_col.release();
    A->jds_val.release();
    A->jds_njd = 0;
    A->jds_built = false;
}

}  // namespace lilac

using namespace lilac;

lilac_status lilac_csr_jds(lilac_csr A, int32_t* perm, int32_t* jd_ptr, int32_t* col_ind, void* vals,
                           int32_t* nzcnt) try {
    if (!A) {
        set_last_error("NULL handle");
        return LILAC_ERR_INVALID_ARG;
    }
    DeviceGuard g(A->device);
    LILAC_TRY(ensure_jds(A, nullptr));
    const size_t n = (size_t)A->rows, nnz = (size_t)A->nnz;
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    auto down = [&](void* h, const lilac::DevBuf& d, size_t bytes) -> lilac_status {
        if (h && bytes) LILAC_CUDA_TRY(cudaMemcpy(h, d.p, bytes, cudaMemcpyDeviceToHost));
        return LILAC_OK;
    };
    LILAC_TRY(down(perm, A->jds_row_slot, sizeof(int32_t) * n));
    LILAC_TRY(down(jd_ptr, A->jds_ptr, sizeof(int32_t) * ((size_t)A->jds_njd + 1)));
    LILAC_TRY(down(col_ind, A->jds_col, sizeof(int32_t) * nnz));
    LILAC_TRY(down(vals, A->jds_val, vsz * nnz));
    LILAC_TRY(down(nzcnt, A->jds_len, sizeof(int32_t) * n));
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}
