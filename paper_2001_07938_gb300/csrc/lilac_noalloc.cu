// lilac_spmv_noalloc: y = A x on CSR arrays the caller already holds on the
// device, without any device allocation.
//
// Who needs it: a caller that must not call cudaMalloc -- for example code
// that runs while another component owns the device memory through its own
// pool and a budget, or a latency-critical loop where cudaMalloc / cudaFree
// (which can synchronise the device) are not acceptable.  Such a caller
// cannot create a handle (lilac_csr_create uploads copies of the matrix), so
// this entry point works on the caller's own arrays and keeps the scratch
// memory of its kernel -- the carry records, per-CTA partial sums and the
// arrival counter of the MERGE kernel -- in one fixed array in device memory
// that every GPU loading the library holds until the process exits.
#include <mutex>

#include "launch.cuh"

namespace lilac {
namespace {

// At most this many CTA ranges per call: the scratch holds one carry record
// and kMaxRed partial sums per CTA, then the arrival counter.
constexpr int kNoAllocMaxCtas = 2048;
constexpr size_t kNoAllocPartialOff = sizeof(MergeCarry) * kNoAllocMaxCtas;
constexpr size_t kNoAllocTicketOff = kNoAllocPartialOff + sizeof(double) * kMaxRed * kNoAllocMaxCtas;
constexpr size_t kNoAllocBytes = kNoAllocTicketOff + 256;  // 82,176 bytes
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};
int g_noalloc_sms[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (in host code its name is only a stand-in) and the SM count.
lilac_status noalloc_setup(int dev, void** addr, int* sms) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("lilac_spmv_noalloc: device id out of range");
        return LILAC_ERR_UNSUPPORTED;
    }
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return LILAC_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        g_noalloc_sms[dev] = n;
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    *sms = g_noalloc_sms[dev];
    return LILAC_OK;
}

template <class T>
lilac_status noalloc_launch(int32_t rows, int64_t nnz, const int32_t* row_ptr, const int32_t* col_ind,
                            const T* vals, const T* x, T* y, unsigned char* scratch, int sms,
                            cudaStream_t s) {
    const int64_t total = (int64_t)rows + nnz;
    const int64_t target = std::min<int64_t>((int64_t)sms * 4, kNoAllocMaxCtas);
    const int64_t per_cta = std::max<int64_t>(kMergeItems, (total + target - 1) / target);
    // per_cta >= ceil(total / target), so G <= target <= kNoAllocMaxCtas: the
    // scratch always has room, whatever the matrix size
    const int64_t G = (total + per_cta - 1) / per_cta;
    unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kNoAllocTicketOff);
    // the arrival counter must start at zero
    LILAC_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    CsrView<T> view{row_ptr, col_ind, vals, rows};
    // CTA start points are searched in the kernel (coords = nullptr)
    spmv_merge_kernel<kMergeThreads, kMergeItems, OpStore<T, T>><<<(unsigned)G, kMergeThreads, 0, s>>>(
        view, nnz, nullptr, per_cta, x, OpStore<T, T>{y},
        reinterpret_cast<double*>(scratch + kNoAllocPartialOff), reinterpret_cast<MergeCarry*>(scratch),
        ticket);
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

}  // namespace
}  // namespace lilac

using namespace lilac;

extern "C" lilac_status lilac_spmv_noalloc(int32_t rows, int32_t ncols, int64_t nnz,
                                           const int32_t* row_ptr, const int32_t* col_ind,
                                           const void* vals, lilac_dtype dtype, const void* x,
                                           void* y, void* stream) try {
    if (rows < 0 || ncols < 0 || nnz < 0 || nnz >= (int64_t(1) << 31) ||
        (int64_t)rows + nnz >= (int64_t(1) << 31) || (rows > 0 && (!row_ptr || !y)) ||
        (nnz > 0 && (!col_ind || !vals || !x)) || (dtype != LILAC_F64 && dtype != LILAC_F32)) {
        set_last_error("invalid argument to lilac_spmv_noalloc (sizes: rows + nnz < 2^31)");
        return LILAC_ERR_INVALID_ARG;
    }
    if (rows == 0) return LILAC_OK;
    int dev = 0;
    LILAC_CUDA_TRY(cudaGetDevice(&dev));
    void* addr = nullptr;
    int sms = 1;
    LILAC_TRY(noalloc_setup(dev, &addr, &sms));
    unsigned char* scratch = static_cast<unsigned char*>(addr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == LILAC_F64)
        return noalloc_launch<double>(rows, nnz, row_ptr, col_ind, static_cast<const double*>(vals),
                                      static_cast<const double*>(x), static_cast<double*>(y),
                                      scratch, sms, s);
    return noalloc_launch<float>(rows, nnz, row_ptr, col_ind, static_cast<const float*>(vals),
                                 static_cast<const float*>(x), static_cast<float*>(y), scratch, sms, s);
} catch (...) {
    return lilac::api_failure();
}
