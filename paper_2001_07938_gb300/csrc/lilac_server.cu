// Request server: a continuous-batching loop over SpMV and CG requests.
//
// The server keeps a pool of registered matrices (host arrays stay with the
// caller).  A matrix is uploaded when a request first needs it and evicted
// (least recently used, not in use) when the device-memory budget would be
// exceeded -- the paper's marshaling (construct on first use, destruct when
// needed, Section 3.3 and Section 4.2) applied to a stream of requests.
// Requests are admitted in arrival order while the budget and the active
// limit allow; each round runs every admitted SpMV request and advances every
// active CG solve by `iters_per_round` iterations; finished requests are
// retired (result copied to the caller's host buffer, latency recorded) and
// their slots and memory go to the next requests in the queue.
//
// Two lanes by size.  Requests on matrices of fewer than kServerLargeNnz
// nonzeros run batched: all single-vector SpMVs in one launch, all CG
// iterations of a round in one captured graph (many small problems, one
// launch).  Requests on larger matrices, and SpMVs of 2..32 vectors, run on
// the matrix's own tuned kernels (lilac_spmv's, lilac_spmm's and lilac_cg's
// iterations, per request one cached graph of a round) on a second stream,
// concurrently with the batched lane; the lane depends on the request alone,
// so a request's result does not depend on the rest of the stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "batch_engine.h"

namespace lilac {

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Caching device allocator with power-of-two size classes (blocks are kept
// for reuse and freed only when the server is destroyed or trimmed).
struct DevicePool {
    std::map<size_t, std::vector<void*>> free_;
    int64_t held = 0;    // bytes obtained from cudaMalloc
    int64_t in_use = 0;  // bytes handed out
    static size_t cls(size_t n) {
        size_t c = 256;
        while (c < n) c <<= 1;
        return c;
    }
    lilac_status get(size_t n, void** out) {
        const size_t c = cls(n);
        auto& v = free_[c];
        if (!v.empty()) {
            *out = v.back();
            v.pop_back();
        } else {
            void* p = nullptr;
            cudaError_t e = cudaMalloc(&p, c);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                set_last_error(std::string("server pool cudaMalloc: ") + cudaGetErrorString(e));
                return LILAC_ERR_OOM;
            }
            held += (int64_t)c;
            *out = p;
        }
        in_use += (int64_t)c;
        return LILAC_OK;
    }
    void put(void* p, size_t n) {
        if (!p) return;
        const size_t c = cls(n);
        free_[c].push_back(p);
        in_use -= (int64_t)c;
    }
    void trim() {
        for (auto& kv : free_)
            for (void* p : kv.second) {
                cudaFree(p);
                held -= (int64_t)kv.first;
            }
        free_.clear();
    }
    ~DevicePool() { trim(); }
};

struct SrvMatrix {
    int32_t rows = 0, ncols = 0;
    int64_t nnz = 0;
    const int32_t* row_ptr = nullptr;
    const int32_t* col_ind = nullptr;
    const double* vals = nullptr;
    lilac_csr h = nullptr;  // resident handle or null
    int64_t bytes = 0;      // device bytes while resident
    int users = 0;          // active requests using it
    uint64_t last_use = 0;
    int64_t uploads = 0;
};

struct SrvRequest {
    lilac_request r;
    double arrival = 0.0;
    double admitted = 0.0;
    int rounds = 0;
    void* ws = nullptr;  // workspace(s) + device vectors
    size_t ws_bytes = 0;
    std::vector<BatchProb> probs;  // one per vector (SpMV) or one (CG); none for multi-vector
    bool started = false;
    bool multi = false;  // SpMV of 2..32 vectors: the multi-vector kernel
    bool large = false;  // single-vector SpMV or CG on a large matrix: its own kernels
    double* xv = nullptr;  // multi: X and Y vector-major, then row-major scratch
    double* yv = nullptr;
    double* scratch = nullptr;
    SoloCg solo;              // large CG: vectors and state in ws
    const double* sb = nullptr;  // large: b (CG) or x (SpMV) on the device
    double* sx = nullptr;        // large: x (CG) or y (SpMV) on the device
    int launched = 0;            // large CG: iterations launched
};

// SpMV requests of this many vectors run through the multi-vector kernel.
constexpr int kServerMultiMin = 2, kServerMultiMax = 32;
// Matrices of at least this many nonzeros run requests on their own kernels.
constexpr int64_t kServerLargeNnz = (int64_t)1 << 19;
constexpr double kServerRuDelta = 0.1;  // reliable-update threshold of precision 2

}  // namespace lilac

using namespace lilac;

struct lilac_server_s {
    int device = 0;
    int sm_count = 1;
    lilac_server_opts o{};
    cudaStream_t stream = nullptr;
    cudaStream_t lane2 = nullptr;  // the large-matrix lane (created with the server)
    cudaEvent_t round_start = nullptr;
    CgState* solo_states = nullptr;  // pinned: the large CG solves' states after a round
    int solo_cap = 0;
    std::vector<SrvMatrix> mats;
    std::deque<SrvRequest*> queue;
    std::vector<SrvRequest*> active;
    std::vector<lilac_completion> done;
    DevicePool pool;
    BatchEngine eng_spmv, eng_cg, eng_start;
    DevBuf states_d;  // compact copy of the CG states of the active solves
    std::vector<CgState> states_h;
    uint64_t clock = 0;
    bool cg_set_changed = true;
    lilac_server_stats_t stats{};
};

namespace lilac {

// Copy the states of the given problems into one contiguous array.
__global__ void gather_states_kernel(const BatchProb* __restrict__ probs, int n,
                                     CgState* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = *probs[i].st;
}

static int64_t resident_bytes(const lilac_server_s* S) {
    int64_t t = 0;
    for (const SrvMatrix& m : S->mats)
        if (m.h) t += m.bytes;
    return t;
}

static int64_t used_bytes(const lilac_server_s* S) { return resident_bytes(S) + S->pool.in_use; }

static int64_t estimate_matrix_bytes(const SrvMatrix& m) {
    // padded arrays, tile list, merge partition and scratch (an upper estimate)
    return (int64_t)m.nnz * 12 + (int64_t)m.rows * 4 + (int64_t)(m.nnz / 2048 + m.rows / 1024 + 16) * 32 +
           (int64_t)8192 * 16 + (1 << 20);
}

// Evict least recently used resident matrices that no active request uses
// (never `keep`) until `need` more bytes fit the budget; false if they cannot.
static bool evict_for(lilac_server_s* S, int64_t need, int keep) {
    while (used_bytes(S) + need > S->o.hbm_budget_bytes) {
        int victim = -1;
        for (int i = 0; i < (int)S->mats.size(); ++i) {
            const SrvMatrix& c = S->mats[i];
            if (i != keep && c.h && c.users == 0 &&
                (victim < 0 || c.last_use < S->mats[victim].last_use))
                victim = i;
        }
        if (victim < 0) return false;
        lilac_csr_destroy(S->mats[victim].h);
        S->mats[victim].h = nullptr;
        S->stats.evictions++;
    }
    return true;
}

// Make matrix `id` resident within the budget; false if it cannot fit now.
static lilac_status make_resident(lilac_server_s* S, int id, bool* ok) {
    SrvMatrix& m = S->mats[id];
    *ok = true;
    if (m.h) return LILAC_OK;
    if (!evict_for(S, estimate_matrix_bytes(m), id)) {
        *ok = false;
        return LILAC_OK;
    }
    LILAC_TRY(lilac_csr_create(m.rows, m.ncols, m.nnz, m.row_ptr, m.col_ind, m.vals, LILAC_F64,
                               LILAC_MEM_HOST, S->o.tune ? 0u : LILAC_CREATE_NO_TUNE, S->stream, &m.h));
    lilac_csr_info_t info;
    lilac_csr_info(m.h, &info);
    m.bytes = info.device_bytes;
    m.uploads++;
    S->stats.uploads++;
    S->stats.upload_bytes += (int64_t)m.nnz * 12 + (int64_t)(m.rows + 1) * 4;
    return LILAC_OK;
}

static int req_prec(const SrvRequest* q) {
    return q->r.kind == LILAC_REQ_CG && q->r.precision == 2 ? BP_F32_RU : BP_F64;
}

static bool req_multi(const SrvRequest* q) {
    return q->r.kind == LILAC_REQ_SPMV && q->r.nvec >= kServerMultiMin && q->r.nvec <= kServerMultiMax;
}

static bool req_large(const lilac_server_s* S, const SrvRequest* q) {
    const SrvMatrix& m = S->mats[q->r.matrix];
    return m.nnz >= kServerLargeNnz && !req_multi(q) &&
           (q->r.kind == LILAC_REQ_CG || q->r.nvec == 1);
}

// Workspace of a request: per-vector problem workspaces + device in/out vectors.
static size_t request_bytes(const lilac_server_s* S, const SrvRequest* q) {
    const SrvMatrix& m = S->mats[q->r.matrix];
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t xb1 = al(sizeof(double) * (size_t)std::max(1, m.ncols));
    const size_t yb1 = al(sizeof(double) * (size_t)std::max(1, m.rows));
    if (req_large(S, q))
        return q->r.kind == LILAC_REQ_SPMV
                   ? xb1 + yb1
                   : al(solo_cg_bytes(m.h, q->r.precision == 2 ? 2 : 0)) + 2 * yb1;
    if (q->r.kind == LILAC_REQ_SPMV) {
        const size_t k = (size_t)q->r.nvec;
        if (req_multi(q))
            return 2 * (al(sizeof(double) * k * (size_t)std::max(1, m.ncols)) +
                        al(sizeof(double) * k * (size_t)std::max(1, m.rows)));
        return k * (al(batch_workspace_bytes(m.h, BK_SPMV, BP_F64)) +
                    al(sizeof(double) * (size_t)std::max(1, m.ncols)) +
                    al(sizeof(double) * (size_t)std::max(1, m.rows)));
    }
    return al(batch_workspace_bytes(m.h, BK_CG, req_prec(q))) + 2 * al(sizeof(double) * (size_t)m.rows);
}

static void retire(lilac_server_s* S, SrvRequest* q, int status, int iters, double rel_res);

static lilac_status admit(lilac_server_s* S) {
    while (!S->queue.empty() && (int)S->active.size() < S->o.max_active) {
        SrvRequest* q = S->queue.front();
        SrvMatrix& m = S->mats[q->r.matrix];
        bool ok = false;
        LILAC_TRY(make_resident(S, q->r.matrix, &ok));
        if (!ok) break;  // wait for memory to be released
        q->multi = req_multi(q);
        q->large = req_large(S, q);
        {
            // what the request's kernels need of the matrix (once per matrix):
            // the batched copy, or the scratch of the matrix's own CG kernels
            if (q->large && q->r.kind == LILAC_REQ_CG && q->r.precision == 0)
                LILAC_TRY(solo_cg_prepare(m.h, 0, S->stream));
            else if (!q->large && !q->multi)
                LILAC_TRY(batch_prepare_layout(m.h, q->r.kind == LILAC_REQ_SPMV ? BK_SPMV : BK_CG,
                                               req_prec(q), S->stream));
            lilac_csr_info_t info;
            lilac_csr_info(m.h, &info);
            m.bytes = info.device_bytes;
        }
        const size_t need = request_bytes(S, q);
        // a mixed-precision solve derives the matrix's FP32 values on first use
        const bool needs_val32 = req_prec(q) == BP_F32_RU && !m.h->val32_valid;
        const int64_t extra = needs_val32 ? (int64_t)m.nnz * 4 + 256 : 0;
        if (!evict_for(S, (int64_t)DevicePool::cls(need) + extra, q->r.matrix)) {
            if (S->active.empty()) {
                // nothing will release memory: the request can never fit
                S->queue.pop_front();
                set_last_error("request larger than the server's device-memory budget");
                q->admitted = now_s();
                m.users++;  // (retire releases one use)
                retire(S, q, LILAC_ERR_BUDGET, 0, 0.0);
                continue;
            }
            S->stats.budget_waits++;
            break;
        }
        if (needs_val32 || (q->large && req_prec(q) == BP_F32_RU)) {
            if (q->large)
                LILAC_TRY(solo_cg_prepare(m.h, 2, S->stream));
            else
                LILAC_TRY(make_val32(m.h, S->stream));
            lilac_csr_info_t info;
            lilac_csr_info(m.h, &info);
            m.bytes = info.device_bytes;
        }
        LILAC_TRY(S->pool.get(need, &q->ws));
        q->ws_bytes = need;
        LILAC_CUDA_TRY(cudaMemsetAsync(q->ws, 0, need, S->stream));
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        unsigned char* w = static_cast<unsigned char*>(q->ws);
        q->probs.clear();
        q->admitted = now_s();
        if (q->large) {
            // SpMV: x | y; CG: the solve's vectors and state | b | x
            const size_t xb = al(sizeof(double) * (size_t)std::max(1, m.ncols));
            const size_t yb = al(sizeof(double) * (size_t)std::max(1, m.rows));
            if (q->r.kind == LILAC_REQ_SPMV) {
                q->sb = reinterpret_cast<const double*>(w);
                q->sx = reinterpret_cast<double*>(w + xb);
                LILAC_CUDA_TRY(cudaMemcpyAsync(w, q->r.in, sizeof(double) * (size_t)m.ncols,
                                               cudaMemcpyHostToDevice, S->stream));
            } else {
                const int prec = q->r.precision == 2 ? 2 : 0;
                const size_t sb = al(solo_cg_bytes(m.h, prec));
                solo_cg_bind(m.h, prec, w, q->solo);
                q->sb = reinterpret_cast<const double*>(w + sb);
                q->sx = reinterpret_cast<double*>(w + sb + yb);
                LILAC_CUDA_TRY(cudaMemcpyAsync(w + sb, q->r.in, sizeof(double) * (size_t)m.rows,
                                               cudaMemcpyHostToDevice, S->stream));
            }
        } else if (q->multi) {
            // X in, then row-major X and Y, then Y out (request_bytes)
            const size_t k = (size_t)q->r.nvec;
            const size_t xb = al(sizeof(double) * k * (size_t)std::max(1, m.ncols));
            const size_t yb = al(sizeof(double) * k * (size_t)std::max(1, m.rows));
            q->xv = reinterpret_cast<double*>(w);
            q->scratch = reinterpret_cast<double*>(w + xb);
            q->yv = reinterpret_cast<double*>(w + 2 * xb + yb);
            LILAC_CUDA_TRY(cudaMemcpyAsync(q->xv, q->r.in, sizeof(double) * k * (size_t)m.ncols,
                                           cudaMemcpyHostToDevice, S->stream));
        } else if (q->r.kind == LILAC_REQ_SPMV) {
            const size_t wsb = al(batch_workspace_bytes(m.h, BK_SPMV, BP_F64));
            const size_t xb = al(sizeof(double) * (size_t)std::max(1, m.ncols));
            const size_t yb = al(sizeof(double) * (size_t)std::max(1, m.rows));
            for (int j = 0; j < q->r.nvec; ++j) {
                double* xd = reinterpret_cast<double*>(w + wsb);
                double* yd = reinterpret_cast<double*>(w + wsb + xb);
                LILAC_CUDA_TRY(cudaMemcpyAsync(xd, q->r.in + (size_t)j * m.ncols,
                                               sizeof(double) * (size_t)m.ncols, cudaMemcpyHostToDevice,
                                               S->stream));
                q->probs.push_back(
                    make_batch_prob(m.h, BK_SPMV, xd, yd, nullptr, nullptr, 0.0, 0, w, BP_F64, 0.0));
                w += wsb + xb + yb;
            }
        } else {
            const size_t wsb = al(batch_workspace_bytes(m.h, BK_CG, req_prec(q)));
            double* bd = reinterpret_cast<double*>(w + wsb);
            double* xd = reinterpret_cast<double*>(w + wsb + al(sizeof(double) * (size_t)m.rows));
            LILAC_CUDA_TRY(cudaMemcpyAsync(bd, q->r.in, sizeof(double) * (size_t)m.rows,
                                           cudaMemcpyHostToDevice, S->stream));
            q->probs.push_back(make_batch_prob(m.h, BK_CG, nullptr, nullptr, bd, xd, q->r.rtol,
                                               q->r.max_iter, w, req_prec(q), 0.1));
            S->cg_set_changed = true;
        }
        m.users++;
        m.last_use = ++S->clock;
        S->queue.pop_front();
        S->active.push_back(q);
    }
    return LILAC_OK;
}

static void retire(lilac_server_s* S, SrvRequest* q, int status, int iters, double rel_res) {
    SrvMatrix& m = S->mats[q->r.matrix];
    lilac_completion c{};
    c.tag = q->r.tag;
    c.status = status;
    c.iters = iters;
    c.rel_res = rel_res;
    c.arrival = q->arrival;
    c.finish = now_s();
    c.admitted = q->admitted;
    c.rounds = q->rounds;
    S->done.push_back(c);
    S->pool.put(q->ws, q->ws_bytes);
    m.users--;
    m.last_use = ++S->clock;
    S->stats.completed++;
    delete q;
}

// The large-matrix lane of a round, on its own stream: multi-vector SpMVs,
// single-vector SpMVs and R iterations of each CG solve on the matrices' own
// kernels, then the solves' states to pinned host memory.
static lilac_status run_lane2(lilac_server_s* S, const std::vector<SrvRequest*>& multi_reqs,
                              const std::vector<SrvRequest*>& big_spmv,
                              const std::vector<SrvRequest*>& big_cg) {
    cudaStream_t s2 = S->lane2;
    // after the admissions' uploads on the server's stream
    LILAC_CUDA_TRY(cudaEventRecord(S->round_start, S->stream));
    LILAC_CUDA_TRY(cudaStreamWaitEvent(s2, S->round_start, 0));
    for (SrvRequest* q : multi_reqs)
        LILAC_TRY(spmm_vectors_device(S->mats[q->r.matrix].h, q->r.nvec, q->xv, q->yv, q->scratch, s2));
    for (SrvRequest* q : big_spmv)
        LILAC_TRY(lilac_spmv(S->mats[q->r.matrix].h, q->sb, q->sx, LILAC_MEM_DEVICE, s2));
    if ((int)big_cg.size() > S->solo_cap) {
        if (S->solo_states) cudaFreeHost(S->solo_states);
        S->solo_states = nullptr;
        S->solo_cap = 0;
        const int cap = std::max(16, 2 * (int)big_cg.size());
        LILAC_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&S->solo_states), sizeof(CgState) * (size_t)cap));
        S->solo_cap = cap;
    }
    for (size_t i = 0; i < big_cg.size(); ++i) {
        SrvRequest* q = big_cg[i];
        lilac_csr h = S->mats[q->r.matrix].h;
        if (!q->started) {
            LILAC_TRY(solo_cg_start(h, q->solo, q->sb, q->sx, q->r.rtol, q->r.max_iter, kServerRuDelta, s2));
            q->started = true;
        }
        // always a whole round: iterations past the end of the solve return at once
        LILAC_TRY(solo_cg_iters(h, q->solo, q->sb, q->sx, S->o.iters_per_round, s2));
        q->launched += S->o.iters_per_round;
        LILAC_CUDA_TRY(cudaMemcpyAsync(&S->solo_states[i], q->solo.W.state.p, sizeof(CgState),
                                       cudaMemcpyDeviceToHost, s2));
    }
    return LILAC_OK;
}

static lilac_status run_round(lilac_server_s* S) {
    cudaStream_t s = S->stream;
    std::vector<SrvRequest*> spmv_reqs, cg_reqs, new_cg, multi_reqs, big_spmv, big_cg;
    for (SrvRequest* q : S->active) {
        q->rounds++;
        if (q->multi)
            multi_reqs.push_back(q);
        else if (q->large)
            (q->r.kind == LILAC_REQ_SPMV ? big_spmv : big_cg).push_back(q);
        else if (q->r.kind == LILAC_REQ_SPMV)
            spmv_reqs.push_back(q);
        else {
            cg_reqs.push_back(q);
            if (!q->started) new_cg.push_back(q);
        }
    }
    const bool lane2 = !multi_reqs.empty() || !big_spmv.empty() || !big_cg.empty();
    if (lane2) LILAC_TRY(run_lane2(S, multi_reqs, big_spmv, big_cg));
    // all SpMV requests in one batched launch
    if (!spmv_reqs.empty()) {
        std::vector<BatchProb> probs;
        for (SrvRequest* q : spmv_reqs) probs.insert(probs.end(), q->probs.begin(), q->probs.end());
        LILAC_TRY(S->eng_spmv.upload(probs, s));
        LILAC_TRY(S->eng_spmv.spmv_phase(s));
    }
    // start new CG solves, then advance all of them
    if (!new_cg.empty()) {
        std::vector<BatchProb> probs;
        for (SrvRequest* q : new_cg) {
            probs.push_back(q->probs[0]);
            q->started = true;
        }
        LILAC_TRY(S->eng_start.upload(probs, s));
        LILAC_TRY(S->eng_start.cg_start(s));
    }
    if (!cg_reqs.empty()) {
        if (S->cg_set_changed) {
            std::vector<BatchProb> probs;
            for (SrvRequest* q : cg_reqs) probs.push_back(q->probs[0]);
            LILAC_TRY(S->eng_cg.upload(probs, s));
            S->cg_set_changed = false;
        }
        LILAC_TRY(S->eng_cg.cg_rounds(S->o.iters_per_round, s));
        const int n = (int)cg_reqs.size();
        if (S->states_d.bytes < sizeof(CgState) * (size_t)n)
            LILAC_TRY(S->states_d.alloc(sizeof(CgState) * (size_t)std::max(64, 2 * n)));
        gather_states_kernel<<<std::max(1, (n + 127) / 128), 128, 0, s>>>(
            S->eng_cg.probs_d.as<BatchProb>(), n, S->states_d.as<CgState>());
        LILAC_CUDA_TRY(cudaGetLastError());
        S->states_h.resize((size_t)n);
        LILAC_CUDA_TRY(cudaMemcpyAsync(S->states_h.data(), S->states_d.p, sizeof(CgState) * (size_t)n,
                                       cudaMemcpyDeviceToHost, s));
    }
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    if (lane2) LILAC_CUDA_TRY(cudaStreamSynchronize(S->lane2));
    S->stats.rounds++;
    // retire: every SpMV request, and the CG solves that are done
    for (SrvRequest* q : spmv_reqs) {
        const SrvMatrix& m = S->mats[q->r.matrix];
        for (int j = 0; j < q->r.nvec; ++j)
            LILAC_CUDA_TRY(cudaMemcpyAsync(q->r.out + (size_t)j * m.rows, q->probs[j].y_out,
                                           sizeof(double) * (size_t)m.rows, cudaMemcpyDeviceToHost, s));
    }
    for (SrvRequest* q : multi_reqs) {
        const SrvMatrix& m = S->mats[q->r.matrix];
        LILAC_CUDA_TRY(cudaMemcpyAsync(q->r.out, q->yv, sizeof(double) * (size_t)q->r.nvec * m.rows,
                                       cudaMemcpyDeviceToHost, s));
    }
    for (SrvRequest* q : big_spmv) {
        const SrvMatrix& m = S->mats[q->r.matrix];
        LILAC_CUDA_TRY(cudaMemcpyAsync(q->r.out, q->sx, sizeof(double) * (size_t)m.rows,
                                       cudaMemcpyDeviceToHost, s));
    }
    // a large solve ends when its state says so (or, as a guard, a round
    // after its iteration limit)
    std::vector<SrvRequest*> finished_big;
    for (size_t i = 0; i < big_cg.size(); ++i) {
        SrvRequest* q = big_cg[i];
        if (S->solo_states[i].done || q->launched > q->r.max_iter) {
            const SrvMatrix& m = S->mats[q->r.matrix];
            LILAC_CUDA_TRY(cudaMemcpyAsync(q->r.out, q->sx, sizeof(double) * (size_t)m.rows,
                                           cudaMemcpyDeviceToHost, s));
            finished_big.push_back(q);
        }
    }
    std::vector<SrvRequest*> finished_cg;
    for (size_t i = 0; i < cg_reqs.size(); ++i)
        if (S->states_h[i].done) {
            const SrvMatrix& m = S->mats[cg_reqs[i]->r.matrix];
            LILAC_CUDA_TRY(cudaMemcpyAsync(cg_reqs[i]->r.out, cg_reqs[i]->probs[0].x,
                                           sizeof(double) * (size_t)m.rows, cudaMemcpyDeviceToHost, s));
            finished_cg.push_back(cg_reqs[i]);
        }
    if (!spmv_reqs.empty() || !multi_reqs.empty() || !big_spmv.empty() || !finished_cg.empty() ||
        !finished_big.empty())
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<SrvRequest*> still;
    for (SrvRequest* q : S->active) {
        if (q->r.kind == LILAC_REQ_SPMV) {
            retire(S, q, LILAC_OK, 0, 0.0);
            continue;
        }
        if (q->large) {
            auto it = std::find(finished_big.begin(), finished_big.end(), q);
            if (it == finished_big.end()) {
                still.push_back(q);
                continue;
            }
            const size_t i = (size_t)(std::find(big_cg.begin(), big_cg.end(), q) - big_cg.begin());
            const CgState& st = S->solo_states[i];
            const double rr = req_prec(q) == BP_F32_RU && st.true_rr >= 0.0 ? st.true_rr : st.rr;
            retire(S, q, st.done ? st.status : LILAC_ERR_NOT_CONVERGED, st.iters,
                   st.bb > 0.0 ? std::sqrt(rr / st.bb) : 0.0);
            continue;
        }
        auto it = std::find(finished_cg.begin(), finished_cg.end(), q);
        if (it != finished_cg.end()) {
            const size_t i = (size_t)(std::find(cg_reqs.begin(), cg_reqs.end(), q) - cg_reqs.begin());
            const CgState& st = S->states_h[i];
            // mixed precision reports its last FP64 residual b - A x
            const double rr = req_prec(q) == BP_F32_RU && st.true_rr >= 0.0 ? st.true_rr : st.rr;
            retire(S, q, st.status, st.iters, st.bb > 0.0 ? std::sqrt(rr / st.bb) : 0.0);
            S->cg_set_changed = true;
        } else {
            still.push_back(q);
        }
    }
    S->active.swap(still);
    return LILAC_OK;
}

}  // namespace lilac

extern "C" {

void lilac_server_opts_default(lilac_server_opts* o) {
    if (!o) return;
    o->hbm_budget_bytes = (int64_t)120 << 30;
    o->max_active = 256;
    o->iters_per_round = 16;
    o->tune = 0;
}

lilac_status lilac_server_create(const lilac_server_opts* opts, void* stream, lilac_server* out) try {
    if (!out) {
        set_last_error("out is NULL");
        return LILAC_ERR_INVALID_ARG;
    }
    *out = nullptr;
    lilac_server_opts o;
    lilac_server_opts_default(&o);
    if (opts) o = *opts;
    if (o.hbm_budget_bytes <= 0 || o.max_active < 1 || o.iters_per_round < 1) {
        set_last_error("invalid lilac_server_opts");
        return LILAC_ERR_INVALID_ARG;
    }
    lilac_server S = new lilac_server_s();
    S->o = o;
    S->stream = static_cast<cudaStream_t>(stream);
    LILAC_CUDA_TRY(cudaGetDevice(&S->device));
    if (cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess ||
        S->sm_count < 1)
        S->sm_count = 1;
    for (BatchEngine* e : {&S->eng_spmv, &S->eng_cg, &S->eng_start}) {
        e->device = S->device;
        e->sm_count = S->sm_count;
    }
    if (cudaStreamCreateWithFlags(&S->lane2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->round_start, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        lilac_server_destroy(S);
        set_last_error("lilac_server_create: stream or event creation failed");
        return LILAC_ERR_CUDA;
    }
    *out = S;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

lilac_status lilac_server_destroy(lilac_server S) try {
    if (!S) return LILAC_OK;
    DeviceGuard g(S->device);
    cudaDeviceSynchronize();
    for (SrvRequest* q : S->active) {
        S->pool.put(q->ws, q->ws_bytes);
        delete q;
    }
    for (SrvRequest* q : S->queue) delete q;
    for (SrvMatrix& m : S->mats)
        if (m.h) lilac_csr_destroy(m.h);
    S->states_d.release();
    if (S->solo_states) cudaFreeHost(S->solo_states);
    if (S->round_start) cudaEventDestroy(S->round_start);
    if (S->lane2) cudaStreamDestroy(S->lane2);
    delete S;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

lilac_status lilac_server_add_matrix(lilac_server S, int32_t rows, int32_t ncols, int64_t nnz,
                                     const int32_t* row_ptr, const int32_t* col_ind,
                                     const double* vals, int32_t* id) try {
    if (!S || !id || rows <= 0 || ncols <= 0 || nnz < 0 || !row_ptr || (nnz > 0 && (!col_ind || !vals))) {
        set_last_error("invalid argument to lilac_server_add_matrix");
        return LILAC_ERR_INVALID_ARG;
    }
    SrvMatrix m;
    m.rows = rows;
    m.ncols = ncols;
    m.nnz = nnz;
    m.row_ptr = row_ptr;
    m.col_ind = col_ind;
    m.vals = vals;
    S->mats.push_back(m);
    *id = (int32_t)S->mats.size() - 1;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

lilac_status lilac_server_submit(lilac_server S, const lilac_request* r) try {
    if (!S || !r || r->matrix < 0 || r->matrix >= (int32_t)S->mats.size() || !r->in || !r->out ||
        (r->kind != LILAC_REQ_SPMV && r->kind != LILAC_REQ_CG) ||
        (r->kind == LILAC_REQ_SPMV && r->nvec < 1) || (r->kind == LILAC_REQ_CG && r->max_iter < 1) ||
        (r->kind == LILAC_REQ_CG && r->precision != 0 && r->precision != 2)) {
        set_last_error("invalid request");
        return LILAC_ERR_INVALID_ARG;
    }
    const SrvMatrix& m = S->mats[r->matrix];
    if (r->kind == LILAC_REQ_CG && m.rows != m.ncols) {
        set_last_error("CG request on a non-square matrix");
        return LILAC_ERR_INVALID_ARG;
    }
    if (estimate_matrix_bytes(m) > S->o.hbm_budget_bytes) {
        set_last_error("matrix larger than the server's device-memory budget");
        return LILAC_ERR_BUDGET;
    }
    SrvRequest* q = new SrvRequest();
    q->r = *r;
    q->arrival = now_s();
    S->queue.push_back(q);
    S->stats.submitted++;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

lilac_status lilac_server_step(lilac_server S, int32_t* active_out) try {
    if (!S) {
        set_last_error("NULL server");
        return LILAC_ERR_INVALID_ARG;
    }
    DeviceGuard g(S->device);
    LILAC_TRY(admit(S));
    if (!S->active.empty()) LILAC_TRY(run_round(S));
    if (active_out) *active_out = (int32_t)(S->active.size() + S->queue.size());
    S->stats.resident_bytes = resident_bytes(S);
    S->stats.pool_bytes = S->pool.held;
    S->stats.queued = (int32_t)S->queue.size();
    S->stats.active = (int32_t)S->active.size();
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

lilac_status lilac_server_poll(lilac_server S, lilac_completion* out, int32_t max, int32_t* n) try {
    if (!S || !n || max < 0 || (max > 0 && !out)) {
        set_last_error("invalid argument to lilac_server_poll");
        return LILAC_ERR_INVALID_ARG;
    }
    const int32_t k = (int32_t)std::min<size_t>((size_t)max, S->done.size());
    for (int32_t i = 0; i < k; ++i) out[i] = S->done[(size_t)i];
    S->done.erase(S->done.begin(), S->done.begin() + k);
    *n = k;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

lilac_status lilac_server_stats(lilac_server S, lilac_server_stats_t* st) try {
    if (!S || !st) {
        set_last_error("invalid argument to lilac_server_stats");
        return LILAC_ERR_INVALID_ARG;
    }
    *st = S->stats;
    return LILAC_OK;
} catch (...) {
    return lilac::api_failure();
}

double lilac_server_now(void) { return now_s(); }

}  // extern "C"
