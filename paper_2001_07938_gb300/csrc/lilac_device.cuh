// Device-side building blocks shared by the library's kernels: inline-PTX
// wrappers for mbarriers and bulk asynchronous copies (sm_90+ / sm_103a),
// bounded waits, deterministic block reductions, and the last-CTA ticket
// that turns per-CTA partial sums into one scalar without a second launch.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lilac {

// Device error word values (written to Scratch::status, read by the host).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1 };
// Test hook word (Scratch::status[1]): the next STAGED launch leaves the first
// tile copy of CTA 0 unissued, so its bounded wait expires.
enum : int { DEV_INJECT_NONE = 0, DEV_INJECT_SKIP_COPY = 2 };

// A bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make mbarrier initialisation visible to the async proxy (bulk copies).
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the mbarrier to complete; false after the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

// L2 eviction policies for bulk copies of data read once per pass.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_policy_evict_normal() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Bulk asynchronous copy global -> this CTA's shared memory, completing
// `bytes` of transaction count on `bar`.  Both addresses 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Streaming 32/64-bit loads that should not displace the gathered vector in L1.
template <class T>
__device__ __forceinline__ T ld_stream(const T* p) {
    return __ldcs(p);
}

// ---------------------------------------------------------------------------
// Reductions.  All orders are fixed by thread index, so a result depends only
// on the grid shape, never on scheduling.

template <int V, class T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <int V>
__device__ __forceinline__ unsigned group_mask(int tid) {
    if constexpr (V >= 32) {
        return 0xffffffffu;
    } else {
        const int lane = tid & 31;
        return ((1u << V) - 1u) << (lane & ~(V - 1));
    }
}

// Sum NR doubles over the block; result valid in thread 0.  `sh` holds
// NR * 32 doubles.  Must be called by all threads of the block.
template <int NR, int THREADS>
__device__ __forceinline__ void block_sum(const double (&v)[NR], double (&out)[NR], double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = THREADS / 32;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        double s = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh[q * 32 + warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            double s = lane < NW ? sh[q * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            out[q] = s;
        }
    }
    __syncthreads();
}

// Sum one value of type T over the block; result valid in every thread.
template <int THREADS, class T>
__device__ __forceinline__ T block_sum_all(T v, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = THREADS / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    T s = T(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sh[w];
    __syncthreads();
    return s;
}

// Scratch memory a launch uses for cross-CTA work.  Counters are zero
// between launches (each user resets what it incremented).
struct Scratch {
    double* partials;         // [max_ctas * kMaxRed] per-CTA partial sums
    double* long_part;        // [num_long_chunks] partial sums of split rows
    double* long_red;         // [num_long_rows * kMaxRed] epilogue sums of split rows
    unsigned int* long_cnt;   // [num_long_rows] arrival counters of split rows
    unsigned int* ticket;     // [1] arrival counter of the grid reduction
    int* status;              // [2] device error word (DEV_*), test hook word (DEV_INJECT_*)
};

constexpr int kMaxRed = 2;

// Publish this CTA's partial sums; the last CTA to arrive adds all partials
// (CTA order, then split-row order) and calls op.finish(tot) in thread 0.
// Must be called by all threads of the block.  `num_long` split rows
// contributed their epilogue sums to s.long_red.
template <int NR, int THREADS, class Op>
__device__ __forceinline__ void grid_reduce_finish(const Op& op, const double (&red)[NR],
                                                   const Scratch& s, int num_long) {
    __shared__ double sh[kMaxRed * 32];
    __shared__ int am_last;
    double tot[NR];
    block_sum<NR, THREADS>(red, tot, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NR; ++q) s.partials[blockIdx.x * NR + q] = tot[q];
        __threadfence();
        const unsigned t = atomicAdd(s.ticket, 1u);
        am_last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += THREADS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] += __ldcg(&s.partials[i * NR + q]);
    }
    for (int i = threadIdx.x; i < num_long; i += THREADS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] += __ldcg(&s.long_red[i * kMaxRed + q]);
    }
    block_sum<NR, THREADS>(acc, tot, sh);
    if (threadIdx.x == 0) {
        op.finish(tot);
        *s.ticket = 0u;
    }
}

}  // namespace lilac
