// lilac_pagerank: PageRank power iteration on the resident transposed link
// matrix (GAP PageRank, the graph kernel of the paper's Section 5 and
// Section 6.1).  One launch per iteration: the SpMV epilogue applies the
// damping and teleport, and sums |y - x| and the next dangling mass in FP64;
// the last CTA turns them into the next teleport term on the device.  The
// dangling set (empty columns) is computed once and cached with the handle,
// like the paper's cached invariants (Section 3.3).
#include <algorithm>
#include <cstring>

#include "launch.cuh"

namespace lilac {

enum { G_PR = 10 };

template <class T>
static lilac_status pagerank_impl(lilac_csr A, T* x, int init_uniform, int iters, double damping,
                                  double* l1_host, cudaStream_t s) {
    const int n = A->rows;
    // dangling set: has_out bit j <=> column j non-empty
    const size_t words = ((size_t)n + 31) / 32;
    if (!A->pr_has_out_valid) {
        LILAC_TRY(A->ws_alloc(A->pr_has_out, sizeof(unsigned) * std::max<size_t>(1, words)));
        LILAC_CUDA_TRY(cudaMemsetAsync(A->pr_has_out.p, 0, A->pr_has_out.bytes, s));
        if (A->nnz > 0) {
            mark_columns_kernel<<<A->sm_count * 8, kVecThreads, 0, s>>>(
                A->nnz, A->col_ind.as<int>(), A->pr_has_out.as<unsigned>());
            LILAC_CUDA_TRY(cudaGetLastError());
        }
        A->pr_has_out_valid = true;
    }
    if (!A->pr_y.p || A->pr_y.bytes < sizeof(T) * (size_t)n)
        LILAC_TRY(A->ws_alloc(A->pr_y, sizeof(T) * (size_t)n));
    if (!A->pr_state.p) LILAC_TRY(A->ws_alloc(A->pr_state, sizeof(PrState)));
    if (!A->pr_l1.p || A->pr_l1.bytes < sizeof(double) * (size_t)std::max(1, iters))
        LILAC_TRY(A->ws_alloc(A->pr_l1, sizeof(double) * (size_t)std::max(1, iters)));
    T* y = A->pr_y.as<T>();
    PrState* st = A->pr_state.as<PrState>();
    double* l1 = A->pr_l1.as<double>();
    const unsigned* has_out = A->pr_has_out.as<unsigned>();
    const T* val = A->val.as<T>();
    using Op = OpPageRank<T, T>;
    LILAC_TRY(prepare_spmv<Op>(A));
    uint64_t dbits;
    std::memcpy(&dbits, &damping, sizeof(dbits));
    const bool prof = A->profiling;
    if (prof) LILAC_TRY(ensure_prof_events(A, iters));
    GraphKey key{G_PR + (init_uniform ? 1 : 0) + (prof ? 2 : 0), x, nullptr, iters, dbits,
                 A->variant, A->vwidth, A->ws_gen};
    LILAC_TRY(run_maybe_graph(A, key, true, s, [&](cudaStream_t cs) -> lilac_status {
        pr_start_kernel<T><<<vec_grid(A, n), kVecThreads, 0, cs>>>(
            n, x, init_uniform, has_out, FinPrStart{st, damping, n}, A->scratch());
        LILAC_CUDA_TRY(cudaGetLastError());
        T* src = x;
        T* dst = y;
        for (int t = 0; t < iters; ++t) {
            Op op{dst, src, has_out, st, l1, T(damping), n};
            if (prof)
                LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * t], cs, cudaEventRecordExternal));
            LILAC_TRY(launch_spmv(A, val, src, op, cs));
            if (prof)
                LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * t + 1], cs, cudaEventRecordExternal));
            std::swap(src, dst);
        }
        if (src != x)
            LILAC_CUDA_TRY(cudaMemcpyAsync(x, src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToDevice, cs));
        return LILAC_OK;
    }));
    if (prof) {
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        int launches = 0;
        double ms = 0.0;
        LILAC_TRY(collect_prof_events(A, iters, &ms, &launches));
        A->prof_ms_acc += ms;
        A->prof_launches_acc += launches;
    }
    if (l1_host && iters > 0) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(l1_host, l1, sizeof(double) * (size_t)iters,
                                       cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return LILAC_OK;
}

}  // namespace lilac

using namespace lilac;

extern "C" lilac_status lilac_pagerank(lilac_csr A, void* x, int32_t init_uniform, int32_t iters,
                                       double damping, double* l1_per_iter, lilac_mem where,
                                       void* stream) try {
    LILAC_TRY(check_handle(A));
    if ((A->rows > 0 && !x) || iters < 0 || !(damping >= 0.0 && damping <= 1.0) ||
        (where != LILAC_MEM_HOST && where != LILAC_MEM_DEVICE)) {
        set_last_error("invalid argument to lilac_pagerank");
        return LILAC_ERR_INVALID_ARG;
    }
    if (A->rows != A->ncols) {
        set_last_error("PageRank needs a square matrix");
        return LILAC_ERR_INVALID_ARG;
    }
    if (A->rows == 0) return LILAC_OK;
    DeviceGuard g(A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    const size_t bytes = vsz * (size_t)A->rows;
    void* xd = x;
    if (where == LILAC_MEM_HOST) {
        if (!A->stage_x.p || A->stage_x.bytes < bytes) LILAC_TRY(A->ws_alloc(A->stage_x, bytes));
        if (!init_uniform) LILAC_CUDA_TRY(cudaMemcpyAsync(A->stage_x.p, x, bytes, cudaMemcpyHostToDevice, s));
        xd = A->stage_x.p;
    }
    if (A->dtype == LILAC_F32)
        LILAC_TRY(pagerank_impl<float>(A, static_cast<float*>(xd), init_uniform, iters, damping,
                                       l1_per_iter, s));
    else
        LILAC_TRY(pagerank_impl<double>(A, static_cast<double*>(xd), init_uniform, iters, damping,
                                        l1_per_iter, s));
    if (where == LILAC_MEM_HOST) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (l1_per_iter || where == LILAC_MEM_HOST) LILAC_TRY(check_device_status(A, s));
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}
