// lilac_spmv: y = A x on the handle's resident matrix (the paper's spmv_csr,
// Section 3.2).  For host vectors the library marshals x in and y out
// through buffers it owns (the CudaRead / CudaWrite roles of Section 3.3),
// allocated on first use and kept with the handle.
#include "launch.cuh"

using namespace lilac;

extern "C" lilac_status lilac_spmv(lilac_csr A, const void* x, void* y, lilac_mem where,
                                   void* stream) try {
    LILAC_TRY(check_handle(A));
    if ((A->rows > 0 && !y) || (A->ncols > 0 && !x) ||
        (where != LILAC_MEM_HOST && where != LILAC_MEM_DEVICE)) {
        set_last_error("invalid argument to lilac_spmv");
        return LILAC_ERR_INVALID_ARG;
    }
    if (A->rows == 0) return LILAC_OK;
    DeviceGuard g(A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    const void* xd = x;
    void* yd = y;
    if (where == LILAC_MEM_HOST) {
        if (!A->stage_x.p && A->ncols > 0) LILAC_TRY(A->ws_alloc(A->stage_x, vsz * (size_t)A->ncols));
        if (!A->stage_y.p) LILAC_TRY(A->ws_alloc(A->stage_y, vsz * (size_t)A->rows));
        if (A->ncols > 0)
            LILAC_CUDA_TRY(cudaMemcpyAsync(A->stage_x.p, x, vsz * (size_t)A->ncols,
                                           cudaMemcpyHostToDevice, s));
        xd = A->stage_x.p;
        yd = A->stage_y.p;
    }
    if (A->dtype == LILAC_F64)
        LILAC_TRY(launch_spmv(A, A->val.as<double>(), static_cast<const double*>(xd),
                              OpStore<double, double>{static_cast<double*>(yd)}, s));
    else
        LILAC_TRY(launch_spmv(A, A->val.as<float>(), static_cast<const float*>(xd),
                              OpStore<float, float>{static_cast<float*>(yd)}, s));
    if (where == LILAC_MEM_HOST) {
        // y and the device error word come back in one synchronization
        int dev_status = DEV_OK;
        LILAC_CUDA_TRY(cudaMemcpyAsync(y, yd, vsz * (size_t)A->rows, cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaMemcpyAsync(&dev_status, A->status.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        if (dev_status != DEV_OK) {
            A->sticky_error = true;
            set_last_error("a device-side bounded wait timed out");
            return LILAC_ERR_TIMEOUT;
        }
    }
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}
