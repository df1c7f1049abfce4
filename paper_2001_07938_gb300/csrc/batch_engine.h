// Host side of the batched engine (lilac_batch.cu): problem descriptors,
// work lists in device memory, captured rounds of CG.
#pragma once

#include <map>
#include <vector>

#include "batch_kernels.cuh"
#include "lilac_impl.h"

namespace lilac {

// Bytes of workspace one problem needs (state, counters, per-item partials,
// split-row scratch, and r, p, q for CG).
size_t batch_workspace_bytes(const lilac_csr_s* A, int kind, int prec);

// prec: BP_F64 or BP_F32_RU (then the handle's FP32 values must exist:
// make_val32); delta: the reliable-update threshold of BP_F32_RU.
BatchProb make_batch_prob(lilac_csr_s* A, int kind, const void* x_in, void* y_out,
                          const double* b, double* x, double rtol, int max_iter, void* ws,
                          int prec, double delta);

// Build, once, the copy the problems of this handle run on in the batch
// (the sliced ELL copy for SELL- or SLAB-tuned handles); call before
// batch_workspace_bytes and make_batch_prob.
lilac_status batch_prepare_layout(lilac_csr_s* A, int kind, int prec, cudaStream_t s);

struct BatchEngine {
    int device = 0;
    int sm_count = 1;
    uint64_t gen = 0;  // bumped when a device buffer is reallocated
    DevBuf probs_d, items_spmv_d, items_vec_d, counts_d;
    std::vector<BatchProb> host_probs;
    std::vector<BatchItem> host_items_spmv, host_items_vec;
    int host_counts[4] = {0, 0, 0, 0};
    bool mixed = false;  // an active CG problem runs in BP_F32_RU
    cudaStream_t capture_stream = nullptr;
    std::map<uint64_t, cudaGraphExec_t> graphs;

    lilac_status ensure(int nprobs, int64_t nspmv, int64_t nvec);
    // Set the active problems (descriptors and work lists); synchronizes s.
    lilac_status upload(const std::vector<BatchProb>& probs, cudaStream_t s);
    int g_spmv = 0, g_vec = 0;  // resident CTAs of the two kernels (0: not yet queried)
    void resident_grids();
    int grid_for(int64_t items, bool spmv);
    lilac_status spmv_phase(cudaStream_t s);
    lilac_status cg_start(cudaStream_t s);
    lilac_status enqueue_rounds(int R, cudaStream_t s, int g1, int g2);
    // R CG iterations of every active problem, as a cached graph.
    lilac_status cg_rounds(int R, cudaStream_t s);
    ~BatchEngine();
};

}  // namespace lilac
