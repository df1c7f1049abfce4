// The CG step kernels: everything of a CG iteration after its SpMV, in one
// launch per iteration (lilac_cg.cu).  Each ends the update (and its r.r)
// with a bounded grid barrier before the direction, so their grids hold at
// most one CTA per SM.
#pragma once

#include "ops.cuh"

namespace lilac {

// One whole CG step after the CG form of the SLAB SpMV, in one launch: the
// update (alpha = r.r / p.q with p.q from the SpMV's CTA sums, added in slot
// order by every CTA; q from the slab partials added in slab order;
// x += alpha p, r -= alpha q), then a grid barrier, then
// r.r from this kernel's CTA sums (every CTA adds them in slot order, so all
// take the same beta = r.r / r.r_old and the same convergence decision) and
// p = r + beta p on the elements the thread updated.  CTA 0 records the step
// in the solver state (iterations, alpha, beta, r.r, done / status) with the
// plain-CG rules of cg_step_kernel, and a breakdown when p.q <= 0 or is not finite.  The
// grid must fit on the GPU at once (at
// most one CTA per SM, see grid_barrier_bounded); a barrier that times out
// leaves DEV_TIMEOUT in the handle's status word.
template <int THREADS>
static __global__ void __launch_bounds__(THREADS, 1)
    cg_step_slabs_kernel(int n, double* __restrict__ x, double* __restrict__ r,
                         double* __restrict__ p, const double* __restrict__ P, int S,
                         const double* __restrict__ pq_parts, int nparts, CgState* st,
                         double* __restrict__ rr_parts, unsigned* bar, int* status) {
    if (cg_done(st)) return;
    const double rr = st->rr;
    const int it = st->iters + 1;
    const int max_iter = st->max_iter;
    const double tol2 = st->tol2;
    const int g0 = blockIdx.x * THREADS + threadIdx.x, gs = gridDim.x * THREADS;
    const bool vec = aligned16(x, r, p, P) && (n & 1) == 0;
    const double2* __restrict__ P2 = reinterpret_cast<const double2*>(P);
    // Held form (every thread has at most kHeld 16-byte vectors, at most
    // kHeldSlabs slabs): the thread's x, r, p and slab partials are loaded
    // before the p.q sum and kept in registers across the grid barrier, so
    // the update and the direction read nothing more: two dependent L2 round
    // trips fewer in a latency-bound step.  Same arithmetic in the same order.
    constexpr int kHeld = 2, kHeldSlabs = 4;
    const int nh = n / 2;
    const bool held = vec && nh <= kHeld * gs && S <= kHeldSlabs;
    double2 xh[kHeld], rh[kHeld], ph[kHeld], qh[kHeld][kHeldSlabs];
    if (held) {
#pragma unroll
        for (int k = 0; k < kHeld; ++k) {
            const int i = g0 + k * gs;
            if (i < nh) {
                xh[k] = reinterpret_cast<const double2*>(x)[i];
                rh[k] = reinterpret_cast<const double2*>(r)[i];
                ph[k] = reinterpret_cast<const double2*>(p)[i];
#pragma unroll
                for (int q = 0; q < kHeldSlabs; ++q)
                    if (q < S) qh[k][q] = P2[(size_t)q * nh + i];
            }
        }
    }
    __shared__ double sh_v;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = (int)threadIdx.x; i < nparts; i += 32) v += __ldcg(pq_parts + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sh_v = v;
    }
    __syncthreads();
    const double pq = sh_v;
    const bool ok = pq > 0.0 && isfinite(pq);
    const double alpha = ok ? rr / pq : 0.0;
    double red[1] = {0.0};
    if (held) {
#pragma unroll
        for (int k = 0; k < kHeld; ++k) {
            const int i = g0 + k * gs;
            if (ok && i < nh) {
                double2 qv = qh[k][0];
#pragma unroll
                for (int q = 1; q < kHeldSlabs; ++q)
                    if (q < S) {
                        qv.x += qh[k][q].x;
                        qv.y += qh[k][q].y;
                    }
                xh[k].x += alpha * ph[k].x;
                xh[k].y += alpha * ph[k].y;
                rh[k].x -= alpha * qv.x;
                rh[k].y -= alpha * qv.y;
                red[0] += rh[k].x * rh[k].x;
                red[0] += rh[k].y * rh[k].y;
                reinterpret_cast<double2*>(x)[i] = xh[k];
                reinterpret_cast<double2*>(r)[i] = rh[k];
            }
        }
    }
    const int nv = (ok && vec && !held) ? nh : 0;
    for (int i = g0; i < nv; i += gs) {
        double2 xv = reinterpret_cast<const double2*>(x)[i], rv = reinterpret_cast<const double2*>(r)[i];
        const double2 pv = reinterpret_cast<const double2*>(p)[i];
        double2 qv = P2[i];
        for (int q = 1; q < S; ++q) {
            const double2 t = P2[(size_t)q * nh + i];
            qv.x += t.x;
            qv.y += t.y;
        }
        xv.x += alpha * pv.x;
        xv.y += alpha * pv.y;
        rv.x -= alpha * qv.x;
        rv.y -= alpha * qv.y;
        red[0] += rv.x * rv.x;
        red[0] += rv.y * rv.y;
        reinterpret_cast<double2*>(x)[i] = xv;
        reinterpret_cast<double2*>(r)[i] = rv;
    }
    // elements left to the scalar loop: all of them when not vectorised
    for (int i = (vec ? 2 * nh : 0) + g0; ok && i < n; i += gs) {
        double qi = P[i];
        for (int q = 1; q < S; ++q) qi += P[(size_t)q * n + i];
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * qi;
        r[i] = ri;
        red[0] += ri * ri;
    }
    {
        __shared__ double sh[32];
        double tot[1];
        block_sum<1, THREADS>(red, tot, sh);
        if (threadIdx.x == 0) rr_parts[blockIdx.x] = tot[0];
    }
    bool skip = false;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        skip = atomicCAS(status + 1, DEV_INJECT_SKIP_BARRIER, DEV_INJECT_NONE) == DEV_INJECT_SKIP_BARRIER;
    if (!grid_barrier_bounded(bar, status, skip)) return;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = (int)threadIdx.x; i < (int)gridDim.x; i += 32) v += __ldcg(rr_parts + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sh_v = v;
    }
    __syncthreads();
    const double rr_new = sh_v;
    bool done = true;
    int code = LILAC_ERR_BREAKDOWN;
    if (ok) {
        if (rr_new == 0.0 || (tol2 >= 0.0 && rr_new <= tol2)) {
            code = LILAC_OK;
        } else if (it >= max_iter) {
            code = tol2 >= 0.0 ? LILAC_ERR_NOT_CONVERGED : LILAC_OK;
        } else {
            done = false;
        }
    }
    const double beta = rr_new / rr;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->pq = pq;
        if (ok) {
            st->alpha = alpha;
            st->iters = it;
            st->beta = beta;
            st->rr = rr_new;
        }
        if (done) {
            st->status = code;
            st->done = 1;
        }
    }
    if (done) return;
    if (held) {
#pragma unroll
        for (int k = 0; k < kHeld; ++k) {
            const int i = g0 + k * gs;
            if (i < nh) {
                double2 pv = ph[k];
                pv.x = rh[k].x + beta * pv.x;
                pv.y = rh[k].y + beta * pv.y;
                reinterpret_cast<double2*>(p)[i] = pv;
            }
        }
        return;
    }
    const int nv2 = vec ? nh : 0;
    for (int i = g0; i < nv2; i += gs) {
        const double2 rv = reinterpret_cast<const double2*>(r)[i];
        double2 pv = reinterpret_cast<const double2*>(p)[i];
        pv.x = rv.x + beta * pv.x;
        pv.y = rv.y + beta * pv.y;
        reinterpret_cast<double2*>(p)[i] = pv;
    }
    for (int i = nv2 * 2 + g0; i < n; i += gs) p[i] = r[i] + beta * p[i];
}

// One whole CG step after the SpMV q = A p (which left alpha in the state),
// in one launch of at most one CTA per SM (all resident), for handles whose
// SpMV writes q:
//   phase 1: u += alpha p, r -= alpha q, r.r per thread (FP64, or compensated
//            FP32 for FP32 vectors), per-CTA sums to rr_parts; u is x, or for
//            RU (FP32 CG with FP64 reliable updates) the FP32 correction d;
//   a bounded grid barrier (grid_barrier_bounded);
//   phase 2: r.r_new from the CTA sums (every CTA adds them in slot order,
//            so all take the same decision), recorded by CTA 0:
//            plain CG: iterations + 1, beta = r.r_new / r.r, r.r = r.r_new;
//            done (OK) when r.r_new = 0 or <= tol2, done at max_iter (OK for
//            a fixed count, else NOT_CONVERGED); RU: a replacement is due
//            when r.r_new fell to delta2 times r.r at the last replacement,
//            is 0 or <= tol2, or the iteration cap is reached; beta and r.r
//            as above either way;
//            then p = r + beta p on the thread's elements, walked backwards
//            so that the r and p it read last -- still in L2, q and u having
//            been streamed with evict-first loads -- come first; for RU,
//            when a replacement is due, also x += d (FP64), d = 0 (the
//            replacement that follows changes r, not the direction).
constexpr int kStepThreads = 1024;
#ifndef LILAC_STEP_UNROLL
#define LILAC_STEP_UNROLL 2
#endif
constexpr int kStepUnroll = LILAC_STEP_UNROLL;

template <class T>
__device__ __forceinline__ typename Vec16<T>::type ld_stream16(const T* a, int i) {
    return __ldcs(reinterpret_cast<const typename Vec16<T>::type*>(a) + i);
}

template <int THREADS, class T, bool RU>
static __global__ void __launch_bounds__(THREADS, 1)
    cg_step_kernel(int n, T* __restrict__ u, double* __restrict__ x64, T* __restrict__ r,
                   T* __restrict__ p, const T* __restrict__ q, CgState* st,
                   double* __restrict__ rr_parts, unsigned* bar, int* status) {
    if (cg_done(st)) return;
    using VT = Vec16<T>;
    using V = typename VT::type;
    constexpr int N = VT::N;
    // every state field this kernel reads, before CTA 0 may write it
    const T alpha = T(st->alpha);
    const double rr_old = st->rr;
    const int it = st->iters + 1;
    const int max_iter = st->max_iter;
    const double tol2 = st->tol2;
    const double ru_bound = RU ? st->delta2 * st->rr_anchor : 0.0;
    typename RedOf<T>::type rr{};
    const int g0 = blockIdx.x * THREADS + threadIdx.x, gs = gridDim.x * THREADS;
    const bool vec = aligned16(u, r, p, q);
    const int nv = vec ? n / N : 0;
    // kStepUnroll vectors of each array in flight per thread, taken in the
    // order of the plain loop (i, i + gs, ...), so the sums are the same
    constexpr int U = kStepUnroll;
    int i0 = g0;
    for (; i0 + (U - 1) * gs < nv; i0 += U * gs) {
        V uv[U], rv[U], pv[U], qv[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * gs;
            uv[k] = ld_stream16(u, i);
            rv[k] = reinterpret_cast<const V*>(r)[i];
            pv[k] = reinterpret_cast<const V*>(p)[i];
            qv[k] = ld_stream16(q, i);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
#pragma unroll
            for (int e = 0; e < N; ++e) {
                VT::set(uv[k], e, VT::get(uv[k], e) + alpha * VT::get(pv[k], e));
                const T ri = VT::get(rv[k], e) - alpha * VT::get(qv[k], e);
                VT::set(rv[k], e, ri);
                red_add_prod(rr, ri, ri);
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int i = i0 + k * gs;
            __stcs(reinterpret_cast<V*>(u) + i, uv[k]);
            reinterpret_cast<V*>(r)[i] = rv[k];
        }
    }
    for (int i = i0; i < nv; i += gs) {
        V uv = ld_stream16(u, i), rv = reinterpret_cast<const V*>(r)[i];
        const V pv = reinterpret_cast<const V*>(p)[i], qv = ld_stream16(q, i);
#pragma unroll
        for (int e = 0; e < N; ++e) {
            VT::set(uv, e, VT::get(uv, e) + alpha * VT::get(pv, e));
            const T ri = VT::get(rv, e) - alpha * VT::get(qv, e);
            VT::set(rv, e, ri);
            red_add_prod(rr, ri, ri);
        }
        __stcs(reinterpret_cast<V*>(u) + i, uv);
        reinterpret_cast<V*>(r)[i] = rv;
    }
    for (int i = nv * N + g0; i < n; i += gs) {
        u[i] += alpha * p[i];
        const T ri = r[i] - alpha * q[i];
        r[i] = ri;
        red_add_prod(rr, ri, ri);
    }
    {
        double red[1] = {red_value(rr)}, tot[1];
        __shared__ double sh[32];
        block_sum<1, THREADS>(red, tot, sh);
        if (threadIdx.x == 0) rr_parts[blockIdx.x] = tot[0];
    }
    bool skip = false;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        skip = atomicCAS(status + 1, DEV_INJECT_SKIP_BARRIER, DEV_INJECT_NONE) == DEV_INJECT_SKIP_BARRIER;
    if (!grid_barrier_bounded(bar, status, skip)) return;
    __shared__ double sh_v;
    if (threadIdx.x < 32) {
        double v = 0.0;
        for (int i = (int)threadIdx.x; i < (int)gridDim.x; i += 32) v += __ldcg(rr_parts + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sh_v = v;
    }
    __syncthreads();
    const double rr_new = sh_v;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    bool direction = true;
    if (RU) {
        const bool due = rr_new <= ru_bound || rr_new == 0.0 || (tol2 >= 0.0 && rr_new <= tol2) ||
                         it >= max_iter;
        if (lead) {
            st->iters = it;
            st->beta = rr_new / rr_old;
            st->rr = rr_new;  // replaced by the new residual's r.r when one is due
            if (due) st->update = 1;
        }
        if (due) {
            // x += d in FP64, d = 0, on the elements this thread updated; the
            // direction below is taken from this iteration's recursive r, and
            // the replacement changes r only (the direction is kept)
            for (int i = g0; i < nv; i += gs)
#pragma unroll
                for (int e = 0; e < N; ++e) {
                    x64[(size_t)i * N + e] += double(u[(size_t)i * N + e]);
                    u[(size_t)i * N + e] = T(0);
                }
            for (int i = nv * N + g0; i < n; i += gs) {
                x64[i] += double(u[i]);
                u[i] = T(0);
            }
        }
    } else {
        const bool conv = rr_new == 0.0 || (tol2 >= 0.0 && rr_new <= tol2);
        const bool cap = it >= max_iter;
        if (lead) {
            st->iters = it;
            st->beta = rr_new / rr_old;
            st->rr = rr_new;
            if (conv) {
                st->done = 1;
                st->status = LILAC_OK;
            } else if (cap) {
                st->done = 1;
                st->status = tol2 >= 0.0 ? LILAC_ERR_NOT_CONVERGED : LILAC_OK;
            }
        }
        direction = !(conv || cap);
    }
    if (!direction) return;
    const T beta = T(rr_new / rr_old);
    for (int i = nv * N + g0; i < n; i += gs) p[i] = r[i] + beta * p[i];
    if (g0 < nv) {
        for (int i = g0 + ((nv - 1 - g0) / gs) * gs; i >= g0; i -= gs) {
            const V rv = reinterpret_cast<const V*>(r)[i];
            V pv = reinterpret_cast<const V*>(p)[i];
#pragma unroll
            for (int e = 0; e < N; ++e) VT::set(pv, e, VT::get(rv, e) + beta * VT::get(pv, e));
            reinterpret_cast<V*>(p)[i] = pv;
        }
    }
}

}  // namespace lilac
