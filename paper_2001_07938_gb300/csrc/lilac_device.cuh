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
// DEV_INJECT_SKIP_BARRIER: in the next fused CG step, CTA 0 does not arrive
// at the grid barrier, so the other CTAs' bounded waits expire.
enum : int { DEV_INJECT_NONE = 0, DEV_INJECT_SKIP_COPY = 2, DEV_INJECT_SKIP_BARRIER = 3 };

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

// Grid-wide barrier for a launch whose CTAs are all resident at once (a grid
// of at most one small CTA per SM): thread 0 of every CTA adds one to bar[0]
// and waits until all gridDim.x have, bounded by kWaitLimitNs of
// %globaltimer; the last CTA to leave resets both counters (bar[1] counts
// departures), so the next launch finds them zero.  A CTA whose wait runs out
// records DEV_TIMEOUT in *status and gets false (its counters stay set until
// the handle's scratch is cleared).  skip (test hook, thread 0): this CTA
// does not arrive, so the others' waits run out.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned* bar, int* status, bool skip) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = skip ? 0 : 1;
        if (ok) {
            __threadfence();
            atomicAdd(bar, 1u);
            const uint64_t t0 = global_timer_ns();
            while (*reinterpret_cast<volatile unsigned*>(bar) < gridDim.x) {
                if (global_timer_ns() - t0 > kWaitLimitNs) {
                    ok = 0;
                    break;
                }
            }
            __threadfence();
        }
        if (ok) {
            if (atomicAdd(bar + 1, 1u) == gridDim.x - 1u) {
                atomicExch(bar, 0u);
                atomicExch(bar + 1, 0u);
            }
        } else {
            atomicExch(status, DEV_TIMEOUT);
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
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

// Sum one value of type T over the block; the result is valid in thread 0
// only, which adds the warps' sums in warp order (the other threads do no
// second-level adds: FP64 adds take the narrow FP64 pipe on GB300).
template <int THREADS, class T>
__device__ __forceinline__ T block_sum_lead(T v, T* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = THREADS / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < NW; ++w) s += sh[w];
    }
    __syncthreads();
    return s;
}

// Scratch memory a launch uses for cross-CTA work.  Counters are zero
// between launches (each user resets what it incremented).
// Per-thread accumulators of the FP64 grid sums.  FP64 work is scarce on
// GB300 (a warp-wide FP64 add or conversion takes an FP64 issue slot), so
// epilogues over FP32 vectors sum per thread in compensated FP32 instead:
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2) keeps the rounding error of every
// addition and TwoProduct (an FMA gives the exact error of a product) that of
// every product, as in the Sum2 / Dot2 algorithms of Ogita, Rump and Oishi
// ("Accurate sum and dot product", SISC 2005): the thread's sum is as
// accurate as one computed in twice the working precision.  The pair becomes
// one FP64 value per thread; sums across threads and CTAs stay FP64.
struct CompF32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float a) {
        const float t = __fadd_rn(s, a);
        const float z = __fsub_rn(t, s);
        c += __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(a, z));
        s = t;
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);      // not contracted into a later add
        const float e = __fmaf_rn(a, b, -p);  // exact: a b = p + e
        add(p);
        c += e;
    }
    // |a - b| exactly as d + e (d = fl(a - b), e its rounding error; |e| <=
    // ulp(d) / 2, so d + e has the sign of d, and d = 0 only when a == b)
    __device__ __forceinline__ void add_absdiff(float a, float b) {
        const float d = __fsub_rn(a, b);
        const float z = __fsub_rn(d, a);
        const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(d, z)), __fsub_rn(-b, z));
        if (d < 0.0f) {
            add(-d);
            c -= e;
        } else {
            add(d);
            c += e;
        }
    }
};

__device__ __forceinline__ double red_value(double v) { return v; }
__device__ __forceinline__ double red_value(const CompF32& v) { return double(v.s) + double(v.c); }

// FP64 accumulation for FP64 vectors, compensated FP32 for FP32 vectors.
template <class T>
struct RedOf {
    using type = double;
};
template <>
struct RedOf<float> {
    using type = CompF32;
};

__device__ __forceinline__ void red_add(double& r, double a) { r += a; }
__device__ __forceinline__ void red_add(CompF32& r, float a) { r.add(a); }
__device__ __forceinline__ void red_add_prod(double& r, double a, double b) { r += a * b; }
__device__ __forceinline__ void red_add_prod(CompF32& r, float a, float b) { r.add_prod(a, b); }
__device__ __forceinline__ void red_add_absdiff(double& r, double a, double b) { r += fabs(a - b); }
__device__ __forceinline__ void red_add_absdiff(CompF32& r, float a, float b) { r.add_absdiff(a, b); }

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

// Like grid_reduce_finish, but a CTA publishes its sums to partial slot
// `slot` (none if negative) and the last CTA adds slots 0 .. nslots - 1 in
// order: the order is fixed even when which CTA fills a slot is not.
template <int NR, int THREADS, class Op>
__device__ __forceinline__ void grid_reduce_slots(const Op& op, const double (&red)[NR],
                                                  const Scratch& s, int slot, int nslots) {
    __shared__ double sh[kMaxRed * 32];
    __shared__ int am_last;
    double tot[NR];
    block_sum<NR, THREADS>(red, tot, sh);
    if (threadIdx.x == 0) {
        if (slot >= 0) {
#pragma unroll
            for (int q = 0; q < NR; ++q) s.partials[slot * NR + q] = tot[q];
        }
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
    for (int i = threadIdx.x; i < nslots; i += THREADS) {
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] += __ldcg(&s.partials[i * NR + q]);
    }
    block_sum<NR, THREADS>(acc, tot, sh);
    if (threadIdx.x == 0) {
        op.finish(tot);
        *s.ticket = 0u;
    }
}

}  // namespace lilac
