// Batched execution of many CSR problems (SpMV, and CG in FP64 or in FP32
// with FP64 reliable updates) in persistent launches: the engine behind
// lilac_batch_* and the request server.
//
// A round of CG is three batched launches (SpMV + p.q; update + r.r;
// direction) over all active problems, five when a mixed-precision problem
// is active (x += d and the FP64 residual, for the problems whose residual
// replacement is due); R rounds are captured once as a CUDA graph whose
// kernels read the problem table and work lists from device buffers, so the
// set of problems can change between replays without a new capture.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch_engine.h"

namespace lilac {

static_assert(kBatchItems == kTileNnz && kBatchRows == kTileRows,
              "batched tiles are the handles' STAGED tiles");

// The layout a problem of this handle runs in: the sliced ELL copy's chunk
// groups when the handle's tuner chose a sliced ELL kernel (SELL, or SLAB,
// whose column slabs need a whole SM each and cannot share a persistent CTA
// with other problems) and the copy holds the values the phase multiplies
// (an FP64 handle's FP32 copy for mixed precision is only in CSR form); the
// STAGED tiles otherwise.
static bool batch_wants_sell(const lilac_csr_s* A, int kind, int prec) {
    if (A->variant != LILAC_VARIANT_SELL && A->variant != LILAC_VARIANT_SLAB) return false;
    if (kind == BK_CG && prec == BP_F32_RU && A->dtype == LILAC_F64) return false;
    return true;
}

static bool batch_uses_sell(const lilac_csr_s* A, int kind, int prec) {
    return batch_wants_sell(A, kind, prec) && A->sell_built;
}

// Build the sliced ELL copy a problem of this handle would run on (once).
lilac_status batch_prepare_layout(lilac_csr_s* A, int kind, int prec, cudaStream_t s) {
    if (batch_wants_sell(A, kind, prec) && !A->sell_built) LILAC_TRY(ensure_sell(A, s));
    return LILAC_OK;
}

static int batch_items(const lilac_csr_s* A, int kind, int prec) {
    return batch_uses_sell(A, kind, prec)
               ? (A->sell_nchunks + kBatchSellChunks - 1) / kBatchSellChunks
               : A->ntiles;
}

size_t batch_workspace_bytes(const lilac_csr_s* A, int kind, int prec) {
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t n = (size_t)std::max(1, A->rows);
    const size_t nchunks = (n + kBatchChunk - 1) / kBatchChunk;
    const bool sell = batch_uses_sell(A, kind, prec);
    const size_t nlong = (size_t)std::max(1, sell ? A->sell_nsplit : A->nlong);
    const size_t nparts = (size_t)std::max(1, sell ? A->sell_npieces : A->nlong_chunks);
    size_t bytes = al(sizeof(CgState)) + al(4 * sizeof(unsigned));
    bytes += al(sizeof(double) * (2 * (size_t)batch_items(A, kind, prec) + nchunks + 1));
    bytes += al(sizeof(double) * nparts);
    bytes += al(sizeof(double) * kMaxRed * nlong);
    bytes += al(sizeof(unsigned) * nlong);
    if (kind == BK_CG) bytes += prec == BP_F32_RU ? 4 * al(sizeof(float) * n) : 3 * al(sizeof(double) * n);
    return bytes;
}

// Fill a problem descriptor from a handle and a workspace block (which must
// hold batch_workspace_bytes and have been zeroed).
BatchProb make_batch_prob(lilac_csr_s* A, int kind, const void* x_in, void* y_out,
                          const double* b, double* x, double rtol, int max_iter, void* ws,
                          int prec, double delta) {
    auto al = [](size_t b_) { return (b_ + 255) & ~size_t(255); };
    unsigned char* w = static_cast<unsigned char*>(ws);
    const size_t n = (size_t)std::max(1, A->rows);
    const size_t nchunks = (n + kBatchChunk - 1) / kBatchChunk;
    const int pr = kind == BK_CG ? prec : BP_F64;
    const bool sell = batch_uses_sell(A, kind, pr);
    BatchProb P{};
    P.row_ptr = A->row_ptr.as<int>();
    P.col_ind = A->col_ind.as<int>();
    P.f32 = A->dtype == LILAC_F32 ? 1 : 0;
    P.val = P.f32 ? nullptr : A->val.as<double>();
    P.val32 = P.f32 ? A->val.as<float>() : A->val32.as<float>();
    P.prec = pr;
    P.delta2 = delta * delta;
    P.tiles = A->tiles.as<TileDesc>();
    P.longs = A->longs.as<LongRow>();
    P.rows = A->rows;
    P.layout = sell ? BL_SELL : BL_TILES;
    P.ntiles = batch_items(A, kind, pr);
    P.nlong = sell ? A->sell_nsplit : A->nlong;
    if (sell) {
        P.scptr = A->sell_cptr.as<int>();
        P.scrow = A->sell_crow.as<int>();
        P.scol = A->sell_col.as<int>();
        P.sval = A->sell_val.p;
        P.ssplits = A->sell_splits.as<int4>();
        P.spiece_split = A->sell_piece_split.as<int>();
        P.snchunks = A->sell_nchunks;
    }
    P.kind = kind;
    P.nchunks = (int)((A->rows + kBatchChunk - 1) / kBatchChunk);
    P.x_in = x_in;
    P.y_out = y_out;
    P.b = b;
    P.x = x;
    P.rtol = rtol;
    P.max_iter = max_iter;
    P.st = reinterpret_cast<CgState*>(w);
    w += al(sizeof(CgState));
    P.cnt = reinterpret_cast<unsigned*>(w);
    w += al(4 * sizeof(unsigned));
    P.part = reinterpret_cast<double*>(w);
    const size_t nlong = (size_t)std::max(1, P.nlong);
    const size_t nparts = (size_t)std::max(1, sell ? A->sell_npieces : A->nlong_chunks);
    w += al(sizeof(double) * (2 * (size_t)P.ntiles + nchunks + 1));
    P.long_part = reinterpret_cast<double*>(w);
    w += al(sizeof(double) * nparts);
    P.long_red = reinterpret_cast<double*>(w);
    w += al(sizeof(double) * kMaxRed * nlong);
    P.long_cnt = reinterpret_cast<unsigned*>(w);
    w += al(sizeof(unsigned) * nlong);
    if (kind == BK_CG && P.prec == BP_F32_RU) {
        float** v[4] = {&P.r32, &P.p32, &P.q32, &P.d32};
        for (float** f : v) {
            *f = reinterpret_cast<float*>(w);
            w += al(sizeof(float) * n);
        }
    } else if (kind == BK_CG) {
        P.r = reinterpret_cast<double*>(w);
        w += al(sizeof(double) * n);
        P.p = reinterpret_cast<double*>(w);
        w += al(sizeof(double) * n);
        P.q = reinterpret_cast<double*>(w);
    }
    return P;
}

lilac_status BatchEngine::ensure(int nprobs, int64_t nspmv, int64_t nvec) {
    auto grow = [&](DevBuf& b, size_t need) -> lilac_status {
        if (b.bytes >= need && b.p) return LILAC_OK;
        ++gen;
        return b.alloc(std::max(need, b.bytes * 2));
    };
    LILAC_TRY(grow(probs_d, sizeof(BatchProb) * (size_t)std::max(1, nprobs)));
    LILAC_TRY(grow(items_spmv_d, sizeof(BatchItem) * (size_t)std::max<int64_t>(1, nspmv)));
    LILAC_TRY(grow(items_vec_d, sizeof(BatchItem) * (size_t)std::max<int64_t>(1, nvec)));
    LILAC_TRY(grow(counts_d, sizeof(int) * 4));
    return LILAC_OK;
}

lilac_status BatchEngine::upload(const std::vector<BatchProb>& probs, cudaStream_t s) {
    std::vector<BatchItem> ispmv, ivec;
    mixed = false;
    for (int i = 0; i < (int)probs.size(); ++i) {
        const BatchProb& P = probs[i];
        mixed = mixed || (P.kind == BK_CG && P.prec == BP_F32_RU);
        for (int t = 0; t < P.ntiles; ++t) ispmv.push_back({i, t});
        if (P.kind == BK_CG)
            for (int c = 0; c < P.nchunks; ++c) ivec.push_back({i, c});
    }
    LILAC_TRY(ensure((int)probs.size(), (int64_t)ispmv.size(), (int64_t)ivec.size()));
    host_probs = probs;
    host_items_spmv.swap(ispmv);
    host_items_vec.swap(ivec);
    host_counts[0] = (int)host_items_spmv.size();
    host_counts[1] = (int)host_items_vec.size();
    if (!probs.empty())
        LILAC_CUDA_TRY(cudaMemcpyAsync(probs_d.p, host_probs.data(), sizeof(BatchProb) * probs.size(),
                                       cudaMemcpyHostToDevice, s));
    if (!host_items_spmv.empty())
        LILAC_CUDA_TRY(cudaMemcpyAsync(items_spmv_d.p, host_items_spmv.data(),
                                       sizeof(BatchItem) * host_items_spmv.size(),
                                       cudaMemcpyHostToDevice, s));
    if (!host_items_vec.empty())
        LILAC_CUDA_TRY(cudaMemcpyAsync(items_vec_d.p, host_items_vec.data(),
                                       sizeof(BatchItem) * host_items_vec.size(),
                                       cudaMemcpyHostToDevice, s));
    LILAC_CUDA_TRY(cudaMemcpyAsync(counts_d.p, host_counts, sizeof(host_counts),
                                   cudaMemcpyHostToDevice, s));
    // the host copies above are read asynchronously: keep them until done
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    return LILAC_OK;
}

// Resident CTAs of the SpMV-phase and vector-phase kernels on the device:
// the grids of their grid-stride loops.
void BatchEngine::resident_grids() {
    if (g_spmv > 0) return;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, batch_spmv_kernel<0>, kBatchThreads, 0) !=
            cudaSuccess || a < 1)
        a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_vec_kernel<1>, kBatchThreads, 0) !=
            cudaSuccess || b < 1)
        b = 1;
    (void)cudaGetLastError();
    g_spmv = sm_count * a;
    g_vec = sm_count * b;
}

int BatchEngine::grid_for(int64_t items, bool spmv) {
    resident_grids();
    return (int)std::max<int64_t>(1, std::min<int64_t>(items, spmv ? g_spmv : g_vec));
}

lilac_status BatchEngine::spmv_phase(cudaStream_t s) {
    if (host_counts[0] == 0) return LILAC_OK;
    batch_spmv_kernel<0><<<grid_for(host_counts[0], true), kBatchThreads, 0, s>>>(
        probs_d.as<BatchProb>(), items_spmv_d.as<BatchItem>(), counts_d.as<int>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

lilac_status BatchEngine::cg_start(cudaStream_t s) {
    if (host_counts[1] == 0) return LILAC_OK;
    batch_vec_kernel<0><<<grid_for(host_counts[1], false), kBatchThreads, 0, s>>>(
        probs_d.as<BatchProb>(), items_vec_d.as<BatchItem>(), counts_d.as<int>() + 1);
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

// One CG iteration of every active problem; graph grids are sized for the
// largest item counts this engine is set up for (items beyond the current
// counts are not touched: the kernels read the counts from the device).
lilac_status BatchEngine::enqueue_rounds(int R, cudaStream_t s, int g1, int g2) {
    for (int r = 0; r < R; ++r) {
        batch_spmv_kernel<0><<<g1, kBatchThreads, 0, s>>>(
            probs_d.as<BatchProb>(), items_spmv_d.as<BatchItem>(), counts_d.as<int>());
        batch_vec_kernel<1><<<g2, kBatchThreads, 0, s>>>(probs_d.as<BatchProb>(),
                                                         items_vec_d.as<BatchItem>(),
                                                         counts_d.as<int>() + 1);
        if (mixed) {
            batch_vec_kernel<3><<<g2, kBatchThreads, 0, s>>>(probs_d.as<BatchProb>(),
                                                             items_vec_d.as<BatchItem>(),
                                                             counts_d.as<int>() + 1);
            batch_spmv_kernel<1><<<g1, kBatchThreads, 0, s>>>(
                probs_d.as<BatchProb>(), items_spmv_d.as<BatchItem>(), counts_d.as<int>());
        }
        batch_vec_kernel<2><<<g2, kBatchThreads, 0, s>>>(probs_d.as<BatchProb>(),
                                                         items_vec_d.as<BatchItem>(),
                                                         counts_d.as<int>() + 1);
    }
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

lilac_status BatchEngine::cg_rounds(int R, cudaStream_t s) {
    if (host_counts[1] == 0) return LILAC_OK;
    // persistent grids: the resident CTAs, independent of the current counts
    resident_grids();
    const uint64_t key = ((uint64_t)R << 33) ^ ((uint64_t)mixed << 32) ^ gen;
    auto it = graphs.find(key);
    if (it == graphs.end()) {
        if (!capture_stream)
            LILAC_CUDA_TRY(cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking));
        LILAC_CUDA_TRY(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
        lilac_status st = enqueue_rounds(R, capture_stream, g_spmv, g_vec);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(capture_stream, &graph);
        if (st != LILAC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        LILAC_CUDA_TRY(e);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        LILAC_CUDA_TRY(e);
        it = graphs.emplace(key, ex).first;
    }
    LILAC_CUDA_TRY(cudaGraphLaunch(it->second, s));
    return LILAC_OK;
}

BatchEngine::~BatchEngine() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    probs_d.release();
    items_spmv_d.release();
    items_vec_d.release();
    counts_d.release();
}

}  // namespace lilac

using namespace lilac;

struct lilac_batch_s {
    BatchEngine eng;
    DevBuf arena;  // workspaces of the current call's problems
};

extern "C" lilac_status lilac_batch_create(lilac_batch* out) try {
    if (!out) {
        set_last_error("out is NULL");
        return LILAC_ERR_INVALID_ARG;
    }
    lilac_batch B = new lilac_batch_s();
    LILAC_CUDA_TRY(cudaGetDevice(&B->eng.device));
    if (cudaDeviceGetAttribute(&B->eng.sm_count, cudaDevAttrMultiProcessorCount, B->eng.device) !=
            cudaSuccess ||
        B->eng.sm_count < 1)
        B->eng.sm_count = 1;
    *out = B;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

extern "C" lilac_status lilac_batch_destroy(lilac_batch B) try {
    if (!B) return LILAC_OK;
    DeviceGuard g(B->eng.device);
    cudaDeviceSynchronize();
    B->arena.release();
    delete B;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

static lilac_status batch_check(lilac_batch B, int32_t count, const lilac_csr* A) {
    if (!B || count < 0 || (count > 0 && !A)) {
        set_last_error("invalid argument to lilac_batch_*");
        return LILAC_ERR_INVALID_ARG;
    }
    for (int i = 0; i < count; ++i) {
        LILAC_TRY(check_handle(A[i]));
        if (A[i]->device != B->eng.device) {
            set_last_error("matrix lives on another device than the batch");
            return LILAC_ERR_INVALID_ARG;
        }
    }
    return LILAC_OK;
}

// Carve zeroed workspaces for the problems out of the batch's arena.
static lilac_status batch_workspaces(lilac_batch B, int32_t count, const lilac_csr* A, int kind,
                                     int prec, std::vector<void*>& ws, cudaStream_t s) {
    std::vector<size_t> sz((size_t)count);
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        sz[i] = batch_workspace_bytes(A[i], kind, prec);
        total += sz[i];
    }
    if (B->arena.bytes < total) {
        ++B->eng.gen;
        LILAC_TRY(B->arena.alloc(std::max(total, B->arena.bytes * 2)));
    }
    if (total) LILAC_CUDA_TRY(cudaMemsetAsync(B->arena.p, 0, total, s));
    ws.resize((size_t)count);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        ws[i] = static_cast<unsigned char*>(B->arena.p) + off;
        off += sz[i];
    }
    return LILAC_OK;
}

extern "C" lilac_status lilac_batch_spmv(lilac_batch B, int32_t count, const lilac_csr* A,
                                         const void* const* x, void* const* y, void* stream) try {
    LILAC_TRY(batch_check(B, count, A));
    if (count > 0 && (!x || !y)) {
        set_last_error("x and y arrays are required");
        return LILAC_ERR_INVALID_ARG;
    }
    if (count == 0) return LILAC_OK;
    DeviceGuard g(B->eng.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int i = 0; i < count; ++i) LILAC_TRY(batch_prepare_layout(A[i], BK_SPMV, BP_F64, s));
    std::vector<void*> ws;
    LILAC_TRY(batch_workspaces(B, count, A, BK_SPMV, BP_F64, ws, s));
    std::vector<BatchProb> probs;
    for (int i = 0; i < count; ++i)
        probs.push_back(make_batch_prob(A[i], BK_SPMV, x[i], y[i], nullptr, nullptr, 0.0, 0, ws[i],
                                        BP_F64, 0.0));
    LILAC_TRY(B->eng.upload(probs, s));
    return B->eng.spmv_phase(s);
} catch (...) {
    return lilac::api_failure();
}

extern "C" lilac_status lilac_batch_cg(lilac_batch B, int32_t count, const lilac_csr* A,
                                       const double* const* b, double* const* x, int32_t max_iter,
                                       double rtol, int32_t precision, lilac_cg_info* infos,
                                       void* stream) try {
    LILAC_TRY(batch_check(B, count, A));
    if ((count > 0 && (!b || !x)) || max_iter < 0 || (precision != 0 && precision != 2)) {
        set_last_error("invalid argument to lilac_batch_cg");
        return LILAC_ERR_INVALID_ARG;
    }
    for (int i = 0; i < count; ++i) {
        if (A[i]->rows != A[i]->ncols || A[i]->rows == 0) {
            set_last_error("lilac_batch_cg needs square, non-empty matrices");
            return LILAC_ERR_INVALID_ARG;
        }
        if (A[i]->dtype == LILAC_F32 && precision != 2) {
            set_last_error("FP32 matrices run batched CG in precision 2 (FP32 CG, FP64 updates)");
            return LILAC_ERR_DTYPE;
        }
    }
    if (count == 0) return LILAC_OK;
    DeviceGuard g(B->eng.device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<void*> ws;
    const int prec = precision == 2 ? BP_F32_RU : BP_F64;
    for (int i = 0; i < count; ++i) {
        if (prec == BP_F32_RU && A[i]->dtype == LILAC_F64) LILAC_TRY(make_val32(A[i], s));
        LILAC_TRY(batch_prepare_layout(A[i], BK_CG, prec, s));
    }
    LILAC_TRY(batch_workspaces(B, count, A, BK_CG, prec, ws, s));
    std::vector<BatchProb> probs;
    for (int i = 0; i < count; ++i)
        probs.push_back(make_batch_prob(A[i], BK_CG, nullptr, nullptr, b[i], x[i], rtol, max_iter, ws[i],
                                        prec, 0.1));
    LILAC_TRY(B->eng.upload(probs, s));
    LILAC_TRY(B->eng.cg_start(s));
    // rounds of R iterations until every problem is done
    const int R = 16;
    std::vector<CgState> hs((size_t)count);
    int done_iters = 0;
    bool all_done = false;
    while (!all_done && done_iters < max_iter) {
        const int r = std::min(R, max_iter - done_iters);
        if (r == R)
            LILAC_TRY(B->eng.cg_rounds(R, s));
        else
            LILAC_TRY(B->eng.enqueue_rounds(r, s, B->eng.grid_for(B->eng.host_counts[0], true),
                                            B->eng.grid_for(B->eng.host_counts[1], false)));
        done_iters += r;
        all_done = true;
        for (int i = 0; i < count; ++i)
            LILAC_CUDA_TRY(cudaMemcpyAsync(&hs[i], probs[i].st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < count; ++i) all_done = all_done && hs[i].done;
    }
    if (!all_done || max_iter == 0) {
        for (int i = 0; i < count; ++i)
            LILAC_CUDA_TRY(cudaMemcpyAsync(&hs[i], probs[i].st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    lilac_status worst = LILAC_OK;
    for (int i = 0; i < count; ++i) {
        if (infos) {
            infos[i] = lilac_cg_info{};
            infos[i].iters = hs[i].iters;
            infos[i].refinements = prec == BP_F32_RU ? hs[i].updates : 0;
            infos[i].status = hs[i].status;
            const double rr = prec == BP_F32_RU && hs[i].true_rr >= 0.0 ? hs[i].true_rr : hs[i].rr;
            infos[i].rel_res = hs[i].bb > 0.0 ? std::sqrt(rr / hs[i].bb) : 0.0;
            // mixed precision: the last FP64 residual b - A x
            infos[i].true_rel_res = prec == BP_F32_RU ? infos[i].rel_res : -1.0;
        }
        if (hs[i].status != LILAC_OK && worst == LILAC_OK) worst = (lilac_status)hs[i].status;
    }
    return worst;
} catch (...) {
    return lilac::api_failure();
}
