// lilac_cg: unpreconditioned conjugate gradient on the resident matrix (the
// NAS CG solver whose SpMV the paper's compiler offloads, Section 2 and
// Section 5), with the dot products and axpys fused around the SpMV and every
// scalar kept on the device, plus the mixed-precision form: FP32 inner CG
// and FP64 iterative refinement.
//
// One iteration is two launches:
//   K1  q = A p, p.q  (SpMV epilogue) -> alpha = rr / p.q
//   K2  x += alpha p, r -= alpha q, r.r -> a bounded grid barrier -> beta,
//       convergence, p = r + beta p (cg_step_kernel; on SLAB handles the
//       SpMV leaves q as slab partials and cg_step_slabs_kernel adds them)
// A solve with a fixed iteration count is replayed as one CUDA graph; with a
// tolerance, graphs of `check_every` iterations are replayed until the
// device flags convergence (kernels after convergence return at once).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "cg_step.cuh"
#include "launch.cuh"

namespace lilac {

__global__ void cg_state_reset_kernel(CgState* st, int max_iter) {
    st->rr = 0.0;
    st->pq = 0.0;
    st->alpha = 0.0;
    st->beta = 0.0;
    st->bb = 0.0;
    st->tol2 = -1.0;
    st->true_rr = -1.0;
    st->iters = 0;
    st->max_iter = max_iter;
    st->done = 0;
    st->status = LILAC_ERR_NOT_CONVERGED;
    st->dir_iter = -1;
}

static lilac_status ensure_cg_work(lilac_csr A, CgWork& W, bool f32) {
    const size_t vsz = f32 ? 4 : 8;
    const size_t n = (size_t)std::max(1, A->rows);
    if (W.r.p && W.n == A->rows) return LILAC_OK;
    W.n = A->rows;
    W.f32 = f32;
    LILAC_TRY(A->ws_alloc(W.r, vsz * n));
    LILAC_TRY(A->ws_alloc(W.p, vsz * n));
    LILAC_TRY(A->ws_alloc(W.q, vsz * n));
    LILAC_TRY(A->ws_alloc(W.state, sizeof(CgState)));
    return LILAC_OK;
}

enum GraphKind {
    G_CG64_FIXED = 1,
    G_CG64_CHUNK = 2,
    G_CG32_CHUNK = 3,
    G_CGRU_CHUNK = 4,
    G_SOLO64 = 5,  // a solve on caller-held memory (the server's lane for large matrices)
    G_SOLORU = 6
};

// Profiling of the SpMV launches (opts->profile): event pairs recorded on the
// launching stream around every SpMV, also inside captured graphs.
struct Prof {
    bool on = false;
    double ms = 0.0;
    int launches = 0;
    int kernels = 0;  // all kernels launched by the solve
};

static lilac_status collect_prof(lilac_csr A, int pairs, Prof& prof) {
    return collect_prof_events(A, pairs, &prof.ms, &prof.launches);
}

// Grid of the fused CG step after a SLAB SpMV: at most one CTA of
// kSlabStepThreads per SM (its grid barrier needs every CTA resident), about
// two elements per thread.  The step is a chain of dependent latencies, so
// more SMs beat fewer barrier arrivals: at n = 75,000, 147 CTAs of 256
// threads took 3.47 ms per 75-iteration solve, 37 of 1,024 threads 3.97 ms.
constexpr int kSlabStepThreads = 256;
static int step_grid(lilac_csr A, int n) {
    const int64_t need = ((int64_t)n + 2 * kSlabStepThreads - 1) / (2 * kSlabStepThreads);
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, A->sm_count));
}

// cg_step_kernel with at most one CTA per SM: CTAs of 1,024 threads when
// every SM gets four elements per thread or more (enough loads in flight for
// HBM), else CTAs of 256 threads with about two elements per thread (more
// SMs for a latency-bound step).
template <class T, bool RU>
static lilac_status launch_cg_step(lilac_csr A, int n, T* u, double* x64, T* r, T* p, const T* q,
                                   CgState* st, cudaStream_t s) {
    unsigned* bar = A->cg_step.as<unsigned>();
    double* rr_parts = reinterpret_cast<double*>(bar + 4);
    const int64_t wide = (int64_t)A->sm_count * kStepThreads * 4;
    if ((int64_t)n >= wide) {
        cg_step_kernel<kStepThreads, T, RU><<<A->sm_count, kStepThreads, 0, s>>>(
            n, u, x64, r, p, q, st, rr_parts, bar, A->status.as<int>());
    } else {
        const int64_t need = ((int64_t)n + 2 * 256 - 1) / (2 * 256);
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(need, A->sm_count));
        cg_step_kernel<256, T, RU><<<g, 256, 0, s>>>(n, u, x64, r, p, q, st, rr_parts, bar,
                                                     A->status.as<int>());
    }
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// The CG step kernels' barrier counters and per-CTA r.r partials.
static lilac_status ensure_cg_step(lilac_csr A, cudaStream_t s) {
    const size_t need = 4 * sizeof(unsigned) + sizeof(double) * (size_t)A->sm_count;
    if (!A->cg_step.p || A->cg_step.bytes < need) {
        LILAC_TRY(A->ws_alloc(A->cg_step, need));
        LILAC_CUDA_TRY(cudaMemsetAsync(A->cg_step.p, 0, A->cg_step.bytes, s));
    }
    return LILAC_OK;
}

// Enqueue `nit` iterations of CG on the work set W (vectors of type T; the
// matrix values `val` of type V).
template <class V, class T>
static lilac_status enqueue_iters(lilac_csr A, const V* val, T* x, CgWork& W, int nit,
                                  cudaStream_t s, bool profile) {
    const int n = A->rows;
    CgState* st = W.state.as<CgState>();
    bool slab_cg = false;
    if constexpr (std::is_same<V, double>::value && std::is_same<T, double>::value)
        slab_cg = slab_cg_active(A, val);
    for (int it = 0; it < nit; ++it) {
        if (profile)
            LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * it], s, cudaEventRecordExternal));
        if constexpr (std::is_same<V, double>::value && std::is_same<T, double>::value) {
            if (slab_cg) {
                // SLAB CG form: q stays as the slab partials and p.q as per-CTA
                // sums; the update adds them and takes alpha itself
                LILAC_TRY(launch_slab_cg(A, W.p.as<double>(), st, s));
                if (profile)
                    LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * it + 1], s,
                                                            cudaEventRecordExternal));
                // the rest of the step (update, r.r, direction) in one launch
                // whose CTAs are all resident: at most one per SM
                unsigned* bar = A->cg_step.as<unsigned>();
                double* rr_parts = reinterpret_cast<double*>(bar + 4);
                cg_step_slabs_kernel<kSlabStepThreads><<<step_grid(A, n), kSlabStepThreads, 0, s>>>(
                    n, x, W.r.as<double>(), W.p.as<double>(), A->slab_P.as<double>(), A->slab_S,
                    A->slab_pq.as<double>(), A->slab_grid, st, rr_parts, bar, A->status.as<int>());
                continue;
            }
        }
        const OpCgPq<V, T> op{W.q.as<T>(), W.p.as<T>(), st};
        LILAC_TRY(launch_spmv(A, val, W.p.as<T>(), op, s));
        if (profile)
            LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * it + 1], s, cudaEventRecordExternal));
        // update, r.r and direction in one launch (a bounded grid barrier)
        LILAC_TRY((launch_cg_step<T, false>(A, n, x, nullptr, W.r.as<T>(), W.p.as<T>(), W.q.as<T>(),
                                             st, s)));
    }
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// Kernels one CG iteration launches.
template <class V, class T>
static int iter_kernels(lilac_csr A, const V* val) {
    if constexpr (std::is_same<V, double>::value && std::is_same<T, double>::value)
        if (slab_cg_active(A, val)) return 2;
    return 1 + spmv_launch_count<OpCgPq<V, T>>(A, val);
}

// What FP64 CG on the handle's values needs before its first (captured)
// iteration: the SpMV's scratch and, for the SLAB CG form, the step kernel's
// barrier counters and r.r partials.
static lilac_status prepare_cg64(lilac_csr A, cudaStream_t s) {
    LILAC_TRY(prepare_spmv<OpCgPq<double, double>>(A));
    if (slab_cg_active(A, A->val.as<double>())) LILAC_TRY(prepare_slab_cg(A));
    return ensure_cg_step(A, s);
}

// Run CG iterations until the device says done: either one graph of
// max_iter iterations (no tolerance) or graphs of `chunk` iterations with a
// host check in between.  `start` enqueues the start of the solve.
template <class V, class T, class Start>
static lilac_status run_cg_loop(lilac_csr A, const V* val, T* x, CgWork& W, int max_iter,
                                bool has_tol, int chunk, bool use_graph, int kind_fixed,
                                int kind_chunk, const void* key_b, Start&& start, cudaStream_t s,
                                CgState* host_state, Prof& prof) {
    LILAC_TRY(prepare_spmv<OpCgPq<V, T>>(A));
    if constexpr (std::is_same<V, double>::value && std::is_same<T, double>::value)
        if (val == A->val.as<double>()) LILAC_TRY(prepare_cg64(A, s));
    LILAC_TRY(ensure_cg_step(A, s));
    const uint64_t pflag = prof.on ? 1 : 0;
    if (!has_tol) {
        if (prof.on) LILAC_TRY(ensure_prof_events(A, max_iter));
        GraphKey key{kind_fixed, key_b, x, max_iter, pflag, A->variant, A->vwidth, A->ws_gen};
        LILAC_TRY(run_maybe_graph(A, key, use_graph, s, [&](cudaStream_t cs) -> lilac_status {
            LILAC_TRY(start(cs));
            return enqueue_iters<V, T>(A, val, x, W, max_iter, cs, prof.on);
        }));
        prof.kernels += 2 + iter_kernels<V, T>(A, val) * max_iter;
        if (prof.on) {
            LILAC_CUDA_TRY(cudaStreamSynchronize(s));
            LILAC_TRY(collect_prof(A, max_iter, prof));
        }
        return LILAC_OK;
    }
    LILAC_TRY(start(s));
    prof.kernels += 2;
    if (prof.on) LILAC_TRY(ensure_prof_events(A, chunk));
    int done_iters = 0;
    while (done_iters < max_iter) {
        const int nit = std::min(chunk, max_iter - done_iters);
        GraphKey key{kind_chunk, key_b, x, nit, pflag, A->variant, A->vwidth, A->ws_gen};
        LILAC_TRY(run_maybe_graph(A, key, use_graph, s, [&](cudaStream_t cs) {
            return enqueue_iters<V, T>(A, val, x, W, nit, cs, prof.on);
        }));
        done_iters += nit;
        prof.kernels += iter_kernels<V, T>(A, val) * nit;
        LILAC_CUDA_TRY(cudaMemcpyAsync(host_state, W.state.p, sizeof(CgState),
                                       cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        if (prof.on) LILAC_TRY(collect_prof(A, nit, prof));
        if (host_state->done) break;
    }
    return LILAC_OK;
}

template <class V>
static lilac_status true_residual(lilac_csr A, const V* val, const double* b, const double* x,
                                  CgState* st, cudaStream_t s) {
    OpResidual<V, RES_TRUE> op{nullptr, nullptr, b, st, 0.0};
    return launch_spmv(A, val, x, op, s);
}

// Plain FP64 CG.
static lilac_status cg_f64(lilac_csr A, const double* b, double* x, const lilac_cg_opts& o,
                           cudaStream_t s, CgState* hs, Prof& prof) {
    if (A->dtype != LILAC_F64) {
        set_last_error("FP64 CG needs an FP64 matrix (use precision 1 for FP32 values)");
        return LILAC_ERR_DTYPE;
    }
    CgWork& W = A->cg64;
    LILAC_TRY(ensure_cg_work(A, W, false));
    const double* val = A->val.as<double>();
    CgState* st = W.state.as<CgState>();
    const int n = A->rows;
    const bool has_tol = o.rtol > 0.0;
    if (o.use_x0) LILAC_TRY(prepare_spmv<OpResidual<double, RES_INIT>>(A));
    auto start = [&](cudaStream_t cs) -> lilac_status {
        cg_state_reset_kernel<<<1, 1, 0, cs>>>(st, o.max_iter);
        if (o.use_x0) {
            OpResidual<double, RES_INIT> op{W.r.as<double>(), W.p.as<double>(), b, st, o.rtol};
            LILAC_TRY(launch_spmv(A, val, x, op, cs));
        } else {
            cg_start_zero_kernel<double, double><<<vec_grid(A, n), kVecThreads, 0, cs>>>(
                n, b, 1.0, x, W.r.as<double>(), W.p.as<double>(), FinCgStart<double>{st, o.rtol},
                A->scratch());
        }
        LILAC_CUDA_TRY(cudaGetLastError());
        return LILAC_OK;
    };
    LILAC_TRY(run_cg_loop<double, double>(A, val, x, W, o.max_iter, has_tol, o.check_every,
                                          o.use_graph != 0, G_CG64_FIXED + (o.use_x0 ? 100 : 0),
                                          G_CG64_CHUNK, b, start, s, hs, prof));
    if (o.true_residual) {
        LILAC_TRY(true_residual(A, val, b, x, st, s));
        prof.kernels += 1;
    }
    return LILAC_OK;
}

// Mixed precision: FP64 residual r = b - A x (handle values), FP32 CG on
// A d = r / ||r|| with FP32 values, x += ||r|| d in FP64; repeat until
// ||r|| <= rtol ||b|| or max_iter refinements.
static lilac_status cg_mixed(lilac_csr A, const double* b, double* x, const lilac_cg_opts& o,
                             cudaStream_t s, CgState* hs, lilac_cg_info* info, Prof& prof) {
    if (A->rows != A->ncols) {
        set_last_error("CG needs a square matrix");
        return LILAC_ERR_INVALID_ARG;
    }
    LILAC_TRY(make_val32(A, s));
    const float* val32 = A->dtype == LILAC_F32 ? A->val.as<float>() : A->val32.as<float>();
    CgWork& W = A->cg32;
    LILAC_TRY(ensure_cg_work(A, W, true));
    const int n = A->rows;
    if (!A->cg_outer_state.p) LILAC_TRY(A->ws_alloc(A->cg_outer_state, sizeof(CgState)));
    if (!A->cg_outer_r.p || A->cg_outer_r.bytes < sizeof(double) * (size_t)std::max(1, n))
        LILAC_TRY(A->ws_alloc(A->cg_outer_r, sizeof(double) * (size_t)std::max(1, n)));
    if (!A->ir_x.p || A->ir_x.bytes < sizeof(float) * (size_t)std::max(1, n))
        LILAC_TRY(A->ws_alloc(A->ir_x, sizeof(float) * (size_t)std::max(1, n)));
    CgState* ost = A->cg_outer_state.as<CgState>();
    double* r64 = A->cg_outer_r.as<double>();
    float* d32 = A->ir_x.as<float>();
    if (!o.use_x0) LILAC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s));
    cg_state_reset_kernel<<<1, 1, 0, s>>>(ost, o.max_iter);
    LILAC_CUDA_TRY(cudaGetLastError());
    prof.kernels += 2;  // make_val32 conversion (first use) is not counted

    int total_inner = 0, refinements = 0;
    CgState outer{};
    lilac_status result = LILAC_ERR_NOT_CONVERGED;
    for (;;) {
        if (A->dtype == LILAC_F64) {
            OpResidual<double, RES_OUTER> op{r64, nullptr, b, ost, o.rtol};
            LILAC_TRY(launch_spmv(A, A->val.as<double>(), x, op, s));
        } else {
            OpResidual<float, RES_OUTER> op{r64, nullptr, b, ost, o.rtol};
            LILAC_TRY(launch_spmv(A, A->val.as<float>(), x, op, s));
        }
        prof.kernels += 1;
        LILAC_CUDA_TRY(cudaMemcpyAsync(&outer, ost, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        if (outer.done) {
            result = LILAC_OK;
            break;
        }
        if (refinements >= o.max_iter) break;
        // inner FP32 solve of A d = r * scale from d = 0
        CgState* ist = W.state.as<CgState>();
        const double scale = outer.scale;
        auto start = [&](cudaStream_t cs) -> lilac_status {
            cg_state_reset_kernel<<<1, 1, 0, cs>>>(ist, o.inner_max_iter);
            cg_start_zero_kernel<float, double><<<vec_grid(A, n), kVecThreads, 0, cs>>>(
                n, r64, scale, d32, W.r.as<float>(), W.p.as<float>(),
                FinCgStart<float>{ist, o.inner_rtol}, A->scratch());
            LILAC_CUDA_TRY(cudaGetLastError());
            return LILAC_OK;
        };
        LILAC_TRY(run_cg_loop<float, float>(A, val32, d32, W, o.inner_max_iter, true,
                                            o.check_every, o.use_graph != 0, G_CG32_CHUNK + 100,
                                            G_CG32_CHUNK, r64, start, s, hs, prof));
        LILAC_CUDA_TRY(cudaMemcpyAsync(hs, ist, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        total_inner += hs->iters;
        if (hs->status == LILAC_ERR_BREAKDOWN && hs->iters == 0) {
            result = LILAC_ERR_BREAKDOWN;
            break;
        }
        ir_apply_kernel<<<vec_grid(A, n), kVecThreads, 0, s>>>(n, x, d32, ost);
        LILAC_CUDA_TRY(cudaGetLastError());
        prof.kernels += 1;
        ++refinements;
    }
    info->iters = total_inner;
    info->refinements = refinements;
    info->status = result;
    info->rel_res = outer.bb > 0.0 ? std::sqrt(outer.rr / outer.bb) : 0.0;
    info->true_rel_res = info->rel_res;  // the outer residual is the true FP64 residual
    return LILAC_OK;
}

// Mixed precision with reliable updates: one FP32 CG (FP32 values and
// vectors, FP64 scalars) whose residual is replaced by the FP64 residual
// b - A x whenever it has fallen by ru_delta, with x accumulated in FP64.
// One iteration is three launches; K3 returns at once unless a replacement
// is due:
//   K1  q = A p, p.q -> alpha            (FP32 values)
//   K2  d += alpha p, r -= alpha q, r.r -> beta, p = r + beta p; when a
//       replacement is due also x += d, d = 0 (FP64 x) and flag it
//   K3  r = float(b - A x), ||b - A x||  (handle values, FP64) -> r.r, convergence
// The replacement changes r and keeps the direction (van der Vorst & Ye).
template <class V>
static lilac_status enqueue_iters_ru(lilac_csr A, const float* val32, const V* val, const double* b,
                                     double* x, float* d, CgWork& W, int nit, cudaStream_t s,
                                     bool profile) {
    const int n = A->rows;
    CgState* st = W.state.as<CgState>();
    float* r = W.r.as<float>();
    float* p = W.p.as<float>();
    float* q = W.q.as<float>();
    for (int it = 0; it < nit; ++it) {
        if (profile)
            LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * it], s, cudaEventRecordExternal));
        LILAC_TRY(launch_spmv(A, val32, p, OpCgPq<float, float>{q, p, st}, s));
        if (profile)
            LILAC_CUDA_TRY(cudaEventRecordWithFlags(A->prof_events[2 * it + 1], s, cudaEventRecordExternal));
        // update, r.r and the direction (and x += d when a replacement is due)
        LILAC_TRY((launch_cg_step<float, true>(A, n, d, x, r, p, q, st, s)));
        LILAC_TRY(launch_spmv(A, val, x, OpResidualRU<V>{r, b, st}, s));
    }
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

template <class V>
static lilac_status cg_mixed_ru_impl(lilac_csr A, const V* val, const double* b, double* x,
                                     const lilac_cg_opts& o, cudaStream_t s, CgState* hs,
                                     lilac_cg_info* info, Prof& prof) {
    LILAC_TRY(make_val32(A, s));
    const float* val32 = A->dtype == LILAC_F32 ? A->val.as<float>() : A->val32.as<float>();
    CgWork& W = A->cg32;
    LILAC_TRY(ensure_cg_work(A, W, true));
    const int n = A->rows;
    if (!A->cg_outer_r.p || A->cg_outer_r.bytes < sizeof(double) * (size_t)std::max(1, n))
        LILAC_TRY(A->ws_alloc(A->cg_outer_r, sizeof(double) * (size_t)std::max(1, n)));
    if (!A->ir_x.p || A->ir_x.bytes < sizeof(float) * (size_t)std::max(1, n))
        LILAC_TRY(A->ws_alloc(A->ir_x, sizeof(float) * (size_t)std::max(1, n)));
    double* r64 = A->cg_outer_r.as<double>();
    float* d = A->ir_x.as<float>();
    CgState* st = W.state.as<CgState>();
    LILAC_TRY(prepare_spmv<OpResidual<V, RES_OUTER>>(A));
    LILAC_TRY(prepare_spmv<OpResidualRU<V>>(A));
    LILAC_TRY(prepare_spmv<OpCgPq<float, float>>(A));
    LILAC_TRY(ensure_cg_step(A, s));
    if (!o.use_x0) LILAC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s));
    cg_state_reset_kernel<<<1, 1, 0, s>>>(st, o.max_iter);
    LILAC_CUDA_TRY(cudaGetLastError());
    {
        OpResidual<V, RES_OUTER> op{r64, nullptr, b, st, o.rtol};
        LILAC_TRY(launch_spmv(A, val, x, op, s));
    }
    const double delta = o.ru_delta;
    ru_start_kernel<<<vec_grid(A, n), kVecThreads, 0, s>>>(n, r64, W.r.as<float>(), W.p.as<float>(), d,
                                                           FinRuStart{st, delta * delta}, A->scratch());
    LILAC_CUDA_TRY(cudaGetLastError());
    prof.kernels += 3;
    const int chunk = o.check_every;
    const uint64_t pflag = prof.on ? 1 : 0;
    if (prof.on) LILAC_TRY(ensure_prof_events(A, chunk));
    LILAC_CUDA_TRY(cudaMemcpyAsync(hs, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    int launched = 0;
    while (!hs->done && launched < o.max_iter) {
        const int nit = std::min(chunk, o.max_iter - launched);
        GraphKey key{G_CGRU_CHUNK, b, x, nit, pflag, A->variant, A->vwidth, A->ws_gen};
        LILAC_TRY(run_maybe_graph(A, key, o.use_graph != 0, s, [&](cudaStream_t cs) {
            return enqueue_iters_ru<V>(A, val32, val, b, x, d, W, nit, cs, prof.on);
        }));
        launched += nit;
        prof.kernels += (1 + spmv_launch_count<OpCgPq<float, float>>(A, val32) +
                         spmv_launch_count<OpResidualRU<V>>(A, val)) * nit;
        LILAC_CUDA_TRY(cudaMemcpyAsync(hs, st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        if (prof.on) LILAC_TRY(collect_prof(A, nit, prof));
    }
    info->iters = hs->iters;
    info->refinements = hs->updates;
    info->status = hs->done ? hs->status : LILAC_ERR_NOT_CONVERGED;
    const double rr = hs->true_rr >= 0.0 ? hs->true_rr : hs->rr;
    info->rel_res = hs->bb > 0.0 ? std::sqrt(rr / hs->bb) : 0.0;
    info->true_rel_res = info->rel_res;  // the last FP64 residual b - A x
    return LILAC_OK;
}

static lilac_status cg_mixed_ru(lilac_csr A, const double* b, double* x, const lilac_cg_opts& o,
                                cudaStream_t s, CgState* hs, lilac_cg_info* info, Prof& prof) {
    if (A->dtype == LILAC_F64)
        return cg_mixed_ru_impl<double>(A, A->val.as<double>(), b, x, o, s, hs, info, prof);
    return cg_mixed_ru_impl<float>(A, A->val.as<float>(), b, x, o, s, hs, info, prof);
}

// --- one solve on caller-held memory ----------------------------------------
// The request server's lane for large matrices: the iterations of lilac_cg
// (FP64, or FP32 CG with FP64 reliable updates) with the handle's tuned
// kernels, R at a time, on vectors and state the caller owns, so that several
// solves may share one handle (run them on one stream: they share its SpMV
// scratch).

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t solo_cg_bytes(const lilac_csr_s* A, int prec) {
    const size_t n = (size_t)std::max(1, A->rows);
    if (prec == 0) return 3 * al256(8 * n) + al256(sizeof(CgState));
    // FP32 r, p, q and correction d; the FP64 residual
    return 4 * al256(4 * n) + al256(sizeof(CgState)) + al256(8 * n);
}

void solo_cg_bind(const lilac_csr_s* A, int prec, void* ws, SoloCg& c) {
    const size_t n = (size_t)std::max(1, A->rows);
    const size_t vb = al256((prec == 0 ? 8 : 4) * n);
    unsigned char* w = static_cast<unsigned char*>(ws);
    c.prec = prec;
    c.W.n = A->rows;
    c.W.f32 = prec != 0;
    c.W.r = DevBuf{w, vb};
    c.W.p = DevBuf{w + vb, vb};
    c.W.q = DevBuf{w + 2 * vb, vb};
    c.W.state = DevBuf{w + 3 * vb, sizeof(CgState)};
    w += 3 * vb + al256(sizeof(CgState));
    c.d = nullptr;
    c.r64 = nullptr;
    if (prec != 0) {
        c.d = reinterpret_cast<float*>(w);
        c.r64 = reinterpret_cast<double*>(w + vb);
    }
}

lilac_status solo_cg_prepare(lilac_csr A, int prec, cudaStream_t s) {
    if (A->dtype != LILAC_F64 || A->rows != A->ncols) {
        set_last_error("solve lane: square FP64 matrices only");
        return LILAC_ERR_INVALID_ARG;
    }
    if (prec == 0) return prepare_cg64(A, s);
    LILAC_TRY(make_val32(A, s));
    LILAC_TRY(prepare_spmv<OpResidual<double, RES_OUTER>>(A));
    LILAC_TRY(prepare_spmv<OpResidualRU<double>>(A));
    LILAC_TRY(prepare_spmv<OpCgPq<float, float>>(A));
    return ensure_cg_step(A, s);
}

lilac_status solo_cg_start(lilac_csr A, SoloCg& c, const double* b, double* x, double rtol,
                           int max_iter, double delta, cudaStream_t s) {
    const int n = A->rows;
    CgState* st = c.W.state.as<CgState>();
    cg_state_reset_kernel<<<1, 1, 0, s>>>(st, max_iter);
    LILAC_CUDA_TRY(cudaGetLastError());
    if (c.prec == 0) {
        cg_start_zero_kernel<double, double><<<vec_grid(A, n), kVecThreads, 0, s>>>(
            n, b, 1.0, x, c.W.r.as<double>(), c.W.p.as<double>(), FinCgStart<double>{st, rtol},
            A->scratch());
    } else {
        LILAC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, s));
        OpResidual<double, RES_OUTER> op{c.r64, nullptr, b, st, rtol};
        LILAC_TRY(launch_spmv(A, A->val.as<double>(), x, op, s));
        ru_start_kernel<<<vec_grid(A, n), kVecThreads, 0, s>>>(
            n, c.r64, c.W.r.as<float>(), c.W.p.as<float>(), c.d, FinRuStart{st, delta * delta},
            A->scratch());
    }
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

lilac_status solo_cg_iters(lilac_csr A, SoloCg& c, const double* b, double* x, int nit,
                           cudaStream_t s) {
    const double* val = A->val.as<double>();
    if (c.prec == 0) {
        GraphKey key{G_SOLO64, c.W.state.p, x, nit, 0, A->variant, A->vwidth, A->ws_gen};
        return run_maybe_graph(A, key, true, s, [&](cudaStream_t cs) {
            return enqueue_iters<double, double>(A, val, x, c.W, nit, cs, false);
        });
    }
    const float* val32 = A->val32.as<float>();
    GraphKey key{G_SOLORU, c.W.state.p, x, nit, 0, A->variant, A->vwidth, A->ws_gen};
    return run_maybe_graph(A, key, true, s, [&](cudaStream_t cs) {
        return enqueue_iters_ru<double>(A, val32, val, b, x, c.d, c.W, nit, cs, false);
    });
}

}  // namespace lilac

using namespace lilac;

extern "C" void lilac_cg_opts_default(lilac_cg_opts* o) {
    if (!o) return;
    o->max_iter = 1000;
    o->rtol = 1e-10;
    o->precision = 0;
    o->inner_rtol = 1e-5;
    o->inner_max_iter = 1000;
    o->use_x0 = 0;
    o->true_residual = 1;
    o->use_graph = 1;
    o->check_every = 32;
    o->profile = 0;
    o->ru_delta = 0.1;
}

extern "C" lilac_status lilac_cg(lilac_csr A, const double* b, double* x, lilac_mem where,
                                 const lilac_cg_opts* opts, lilac_cg_info* info, void* stream) try {
    LILAC_TRY(check_handle(A));
    lilac_cg_opts o;
    lilac_cg_opts_default(&o);
    if (opts) o = *opts;
    if ((A->rows > 0 && (!b || !x)) || o.max_iter < 0 || o.precision < 0 || o.precision > 2 ||
        o.check_every < 1 || (where != LILAC_MEM_HOST && where != LILAC_MEM_DEVICE) ||
        (o.precision == 1 && (o.inner_max_iter < 1 || !(o.inner_rtol > 0.0))) ||
        (o.precision == 2 && !(o.ru_delta > 0.0 && o.ru_delta < 1.0))) {
        set_last_error("invalid argument to lilac_cg");
        return LILAC_ERR_INVALID_ARG;
    }
    if (A->rows != A->ncols) {
        set_last_error("CG needs a square matrix");
        return LILAC_ERR_INVALID_ARG;
    }
    lilac_cg_info local{};
    if (A->rows == 0) {
        if (info) *info = lilac_cg_info{0, 0, LILAC_OK, 0, 0.0, 0.0, 0.0, 0, 0};
        return LILAC_OK;
    }
    DeviceGuard g(A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = A->rows;
    const double* bd = b;
    double* xd = x;
    if (where == LILAC_MEM_HOST) {
        if (!A->ir_b.p) LILAC_TRY(A->ws_alloc(A->ir_b, sizeof(double) * (size_t)n));
        if (!A->stage_y.p || A->stage_y.bytes < sizeof(double) * (size_t)n)
            LILAC_TRY(A->ws_alloc(A->stage_y, sizeof(double) * (size_t)n));
        LILAC_CUDA_TRY(cudaMemcpyAsync(A->ir_b.p, b, sizeof(double) * (size_t)n,
                                       cudaMemcpyHostToDevice, s));
        if (o.use_x0)
            LILAC_CUDA_TRY(cudaMemcpyAsync(A->stage_y.p, x, sizeof(double) * (size_t)n,
                                           cudaMemcpyHostToDevice, s));
        bd = A->ir_b.as<double>();
        xd = A->stage_y.as<double>();
    }
    CgState hs{};
    lilac_status st;
    Prof prof;
    prof.on = (o.profile != 0 && info != nullptr) || A->profiling;
    if (o.precision == 0) {
        st = cg_f64(A, bd, xd, o, s, &hs, prof);
        if (st == LILAC_OK && (info || o.rtol > 0.0 || where == LILAC_MEM_HOST)) {
            LILAC_CUDA_TRY(cudaMemcpyAsync(&hs, A->cg64.state.p, sizeof(CgState),
                                           cudaMemcpyDeviceToHost, s));
            LILAC_CUDA_TRY(cudaStreamSynchronize(s));
            local.iters = hs.iters;
            local.refinements = 0;
            local.status = hs.status;
            local.rel_res = hs.bb > 0.0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
            local.true_rel_res = (o.true_residual && hs.true_rr >= 0.0 && hs.bb > 0.0)
                                     ? std::sqrt(hs.true_rr / hs.bb)
                                     : (o.true_residual && hs.bb == 0.0 ? 0.0 : -1.0);
        }
    } else if (o.precision == 1) {
        st = cg_mixed(A, bd, xd, o, s, &hs, &local, prof);
    } else {
        st = cg_mixed_ru(A, bd, xd, o, s, &hs, &local, prof);
    }
    if (st != LILAC_OK) return st;
    if (A->profiling) {
        A->prof_ms_acc += prof.ms;
        A->prof_launches_acc += prof.launches;
    }
    local.spmv_ms = prof.ms;
    local.spmv_launches = prof.launches;
    local.kernel_launches = prof.kernels;
    if (where == LILAC_MEM_HOST) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(x, xd, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    if (info || o.rtol > 0.0 || o.precision != 0) LILAC_TRY(check_device_status(A, s));
    if (info) *info = local;
    if (info || o.rtol > 0.0 || o.precision != 0) {
        if (local.status == LILAC_ERR_BREAKDOWN || local.status == LILAC_ERR_NOT_CONVERGED)
            return (lilac_status)local.status;
    }
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}
