// lilac_spmm: Y = A X for k right-hand sides at once (k <= 32) on the
// resident matrix: each nonzero is streamed from HBM once and used for all k
// vectors, so the matrix bytes per vector fall by k.
//
// One warp per row (grid-stride).  The warp's lanes are (group g, vector j)
// pairs with K lanes per group (K = k rounded up to a power of two): each
// group takes every (32/K)-th nonzero of the row, four at a time in flight,
// its K lanes read the k
// adjacent values X[c][0..k) of row-major X (one coalesced access per
// nonzero), and the groups' sums are added by shuffles at the end of the row.
// Column-major X / Y (k separate vectors) are transposed through device
// scratch around the kernel.
#include <algorithm>

#include "launch.cuh"

namespace lilac {

template <int K, class T>
__global__ void __launch_bounds__(256)
    spmm_rows_kernel(CsrView<T> A, int k, const T* __restrict__ X, T* __restrict__ Y) {
    constexpr int G = 32 / K;  // nonzeros in flight per warp step
    const int lane = threadIdx.x & 31;
    const int g = lane / K, j = lane % K;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    const bool live = j < k;
    for (int r = warp; r < A.rows; r += nwarps) {
        const int kb = __ldg(A.row_ptr + r), ke = __ldg(A.row_ptr + r + 1);
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int q = kb + g;
        // four nonzeros per group in flight
        for (; q + 3 * G < ke; q += 4 * G) {
            int c[4];
            T v[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = ld_stream(A.col_ind + q + u * G);
                v[u] = ld_stream(A.val + q + u * G);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = live ? __ldg(X + (size_t)c[u] * k + j) : T(0);
            s0 += v[0] * xv[0];
            s1 += v[1] * xv[1];
            s2 += v[2] * xv[2];
            s3 += v[3] * xv[3];
        }
        for (; q < ke; q += G) {
            const int c0 = ld_stream(A.col_ind + q);
            const T v0 = ld_stream(A.val + q);
            s0 += v0 * (live ? __ldg(X + (size_t)c0 * k + j) : T(0));
        }
        T s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int off = K; off < 32; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (g == 0 && live) Y[(size_t)r * k + j] = s;
    }
}

// out[i * k + j] = in[j * n + i] (to_rows) or the inverse.
template <class T>
__global__ void spmm_transpose_kernel(int n, int k, const T* __restrict__ in, T* __restrict__ out,
                                      bool to_rows) {
    const int64_t total = (int64_t)n * k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / k, j = t % k;
        if (to_rows)
            out[t] = in[j * n + i];
        else
            out[j * n + i] = in[t];
    }
}

template <class T>
static lilac_status spmm_launch(lilac_csr A, int k, const T* X, T* Y, cudaStream_t s) {
    CsrView<T> view{A->row_ptr.as<int>(), A->col_ind.as<int>(), A->val.as<T>(), A->rows};
    const int64_t need = ((int64_t)A->rows * 32 + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)A->sm_count * 8));
    if (k <= 1)
        spmm_rows_kernel<1, T><<<grid, 256, 0, s>>>(view, k, X, Y);
    else if (k <= 2)
        spmm_rows_kernel<2, T><<<grid, 256, 0, s>>>(view, k, X, Y);
    else if (k <= 4)
        spmm_rows_kernel<4, T><<<grid, 256, 0, s>>>(view, k, X, Y);
    else if (k <= 8)
        spmm_rows_kernel<8, T><<<grid, 256, 0, s>>>(view, k, X, Y);
    else if (k <= 16)
        spmm_rows_kernel<16, T><<<grid, 256, 0, s>>>(view, k, X, Y);
    else
        spmm_rows_kernel<32, T><<<grid, 256, 0, s>>>(view, k, X, Y);
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

template <class T>
static lilac_status spmm_impl(lilac_csr A, const T* X, T* Y, int k, int layout, lilac_mem where,
                              cudaStream_t s) {
    const size_t xn = (size_t)A->ncols * k, yn = (size_t)A->rows * k;
    const T* xd = X;
    T* yd = Y;
    const bool host = where == LILAC_MEM_HOST;
    const bool rows_layout = layout == LILAC_LAYOUT_ROWS;
    // device buffers: staged X / Y (host calls) and row-major scratch (column-major calls)
    if (host || !rows_layout) {
        const size_t need = sizeof(T) * (xn + yn) * (rows_layout ? 1 : 2);
        if (!A->spmm_buf.p || A->spmm_buf.bytes < need) LILAC_TRY(A->ws_alloc(A->spmm_buf, need));
    }
    T* base = A->spmm_buf.as<T>();
    T* xs = base;          // X as given, on the device (host calls)
    T* ys = base + xn;     // Y as returned, on the device (host calls)
    T* xr = rows_layout ? nullptr : base + xn + yn;  // row-major X
    T* yr = rows_layout ? nullptr : xr + xn;          // row-major Y
    if (host) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(xs, X, sizeof(T) * xn, cudaMemcpyHostToDevice, s));
        xd = xs;
        yd = ys;
    }
    const int tg = A->sm_count * 8;
    if (rows_layout) {
        LILAC_TRY(spmm_launch<T>(A, k, xd, yd, s));
    } else {
        spmm_transpose_kernel<T><<<tg, 256, 0, s>>>(A->ncols, k, xd, xr, true);
        LILAC_CUDA_TRY(cudaGetLastError());
        LILAC_TRY(spmm_launch<T>(A, k, xr, yr, s));
        spmm_transpose_kernel<T><<<tg, 256, 0, s>>>(A->rows, k, yr, yd, false);
        LILAC_CUDA_TRY(cudaGetLastError());
    }
    if (host) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(Y, yd, sizeof(T) * yn, cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LILAC_OK;
}

// Y = A X for k (<= 32) FP64 vectors given and returned vector-major on the
// device (X: k x ncols, Y: k x rows), through caller-held row-major scratch
// (k x ncols then k x rows doubles): the server's multi-vector requests.
lilac_status spmm_vectors_device(lilac_csr A, int k, const double* Xv, double* Yv, double* scratch,
                                 cudaStream_t s) {
    double* xr = scratch;
    double* yr = scratch + (size_t)k * A->ncols;
    const int tg = A->sm_count * 8;
    spmm_transpose_kernel<double><<<tg, 256, 0, s>>>(A->ncols, k, Xv, xr, true);
    LILAC_CUDA_TRY(cudaGetLastError());
    LILAC_TRY(spmm_launch<double>(A, k, xr, yr, s));
    spmm_transpose_kernel<double><<<tg, 256, 0, s>>>(A->rows, k, yr, Yv, false);
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

}  // namespace lilac

using namespace lilac;

extern "C" lilac_status lilac_spmm(lilac_csr A, const void* X, void* Y, int32_t k, int32_t layout,
                                   lilac_mem where, void* stream) try {
    LILAC_TRY(check_handle(A));
    if (k < 1 || k > 32 || (layout != LILAC_LAYOUT_ROWS && layout != LILAC_LAYOUT_VECTORS) ||
        (where != LILAC_MEM_HOST && where != LILAC_MEM_DEVICE) ||
        (A->rows > 0 && !Y) || (A->ncols > 0 && !X)) {
        set_last_error("invalid argument to lilac_spmm (k must be 1..32)");
        return LILAC_ERR_INVALID_ARG;
    }
    if (A->rows == 0) return LILAC_OK;
    DeviceGuard g(A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (A->dtype == LILAC_F64)
        LILAC_TRY(spmm_impl<double>(A, static_cast<const double*>(X), static_cast<double*>(Y), k,
                                    layout, where, s));
    else
        LILAC_TRY(spmm_impl<float>(A, static_cast<const float*>(X), static_cast<float*>(Y), k,
                                   layout, where, s));
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}
