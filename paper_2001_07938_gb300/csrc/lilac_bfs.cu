// lilac_bfs: breadth-first search levels as repeated masked boolean SpMVs on
// the resident transposed adjacency matrix (row v lists the sources u of the
// edges u -> v) -- the GAP BFS kernel of the paper's Section 5, whose
// bottom-up loop over each vertex's in-neighbours has the shape of SpMV.
//
// Level L -> L+1 is one launch over all nonzeros (v, u): an unvisited v
// whose in-neighbour u is at level L joins level L+1.  The nonzeros are taken
// in order, perfectly balanced whatever the row lengths (a row index per
// nonzero is derived once from row_ptr and cached with the handle); a
// visited row costs only its row indices.  A vertex is claimed by
// compare-and-swap, so the count of new vertices is exact and the levels are
// the unique BFS levels.  The launch that finds no new vertex marks the
// search done; later launches return at once.  Levels run in captured
// graphs of kBfsChunk launches with one host check between graphs.
#include <algorithm>

#include "launch.cuh"

namespace lilac {

enum { G_BFS = 20 };
constexpr int kBfsChunk = 8;

struct BfsState {
    int cur;   // deepest level assigned so far
    int done;  // 1: the last launch found no new vertex
    int pad[2];
};

struct FinBfs {
    BfsState* st;
    __device__ void finish(const double* tot) const {
        if (tot[0] == 0.0)
            st->done = 1;
        else
            st->cur += 1;
    }
};

static __global__ void __launch_bounds__(kVecThreads)
    bfs_rows_kernel(int rows, const int* __restrict__ row_ptr, int* __restrict__ row_of) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)kVecThreads + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * (int64_t)kVecThreads) >> 5);
    for (int r = warp; r < rows; r += nwarps)
        for (int k = row_ptr[r] + lane; k < row_ptr[r + 1]; k += 32) row_of[k] = r;
}

static __global__ void __launch_bounds__(kVecThreads)
    bfs_init_kernel(int n, int* __restrict__ level, int source, BfsState* st) {
    for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < n; i += gridDim.x * kVecThreads)
        level[i] = i == source ? 0 : -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->cur = 0;
        st->done = 0;
    }
}

// One level: level values only change from -1 to L+1 during the launch, so a
// stale read can neither create a false L nor hide a real one.
static __global__ void __launch_bounds__(kVecThreads)
    bfs_pull_kernel(int64_t nnz, const int* __restrict__ row_of, const int* __restrict__ col,
                    int* level, BfsState* st, Scratch s) {
    if (*reinterpret_cast<const volatile int*>(&st->done)) return;
    const int L = st->cur;
    double red[1] = {0.0};
    for (int64_t k = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * kVecThreads) {
        const int v = ld_stream(row_of + k);
        if (level[v] != -1) continue;
        const int u = ld_stream(col + k);
        if (level[u] == L && atomicCAS(level + v, -1, L + 1) == -1) red[0] += 1.0;
    }
    grid_reduce_finish<1, kVecThreads>(FinBfs{st}, red, s, 0);
}

static lilac_status bfs_impl(lilac_csr A, int source, int* level, int* depth, cudaStream_t s) {
    const int n = A->rows;
    if (!A->bfs_row.p && A->nnz > 0) {
        LILAC_TRY(A->ws_alloc(A->bfs_row, sizeof(int32_t) * (size_t)A->nnz));
        bfs_rows_kernel<<<A->sm_count * 8, kVecThreads, 0, s>>>(n, A->row_ptr.as<int>(),
                                                                  A->bfs_row.as<int>());
        LILAC_CUDA_TRY(cudaGetLastError());
    }
    if (!A->bfs_state.p) LILAC_TRY(A->ws_alloc(A->bfs_state, sizeof(BfsState)));
    BfsState* st = A->bfs_state.as<BfsState>();
    bfs_init_kernel<<<vec_grid(A, n), kVecThreads, 0, s>>>(n, level, source, st);
    LILAC_CUDA_TRY(cudaGetLastError());
    BfsState hs{};
    if (A->nnz > 0) {
        const int grid = A->sm_count * 8;
        for (int launched = 0; launched <= n; launched += kBfsChunk) {
            GraphKey key{G_BFS, level, nullptr, kBfsChunk, 0, 0, 0, A->ws_gen};
            LILAC_TRY(run_maybe_graph(A, key, true, s, [&](cudaStream_t cs) -> lilac_status {
                for (int i = 0; i < kBfsChunk; ++i)
                    bfs_pull_kernel<<<grid, kVecThreads, 0, cs>>>(A->nnz, A->bfs_row.as<int>(),
                                                                  A->col_ind.as<int>(), level, st,
                                                                  A->scratch());
                LILAC_CUDA_TRY(cudaGetLastError());
                return LILAC_OK;
            }));
            LILAC_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(BfsState), cudaMemcpyDeviceToHost, s));
            LILAC_CUDA_TRY(cudaStreamSynchronize(s));
            if (hs.done) break;
        }
    }
    if (depth) *depth = hs.cur + 1;
    return LILAC_OK;
}

}  // namespace lilac

using namespace lilac;

extern "C" lilac_status lilac_bfs(lilac_csr A, int32_t source, int32_t* level, lilac_mem where,
                                  int32_t* depth, void* stream) try {
    LILAC_TRY(check_handle(A));
    if (A->rows != A->ncols) {
        set_last_error("BFS needs a square matrix");
        return LILAC_ERR_INVALID_ARG;
    }
    if (source < 0 || source >= A->rows || !level ||
        (where != LILAC_MEM_HOST && where != LILAC_MEM_DEVICE)) {
        set_last_error("invalid argument to lilac_bfs (source must be a vertex, level non-NULL)");
        return LILAC_ERR_INVALID_ARG;
    }
    DeviceGuard g(A->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(int32_t) * (size_t)A->rows;
    int* ld = level;
    if (where == LILAC_MEM_HOST) {
        if (!A->bfs_level.p || A->bfs_level.bytes < bytes) LILAC_TRY(A->ws_alloc(A->bfs_level, bytes));
        ld = A->bfs_level.as<int>();
    }
    LILAC_TRY(bfs_impl(A, source, ld, depth, s));
    if (where == LILAC_MEM_HOST) {
        LILAC_CUDA_TRY(cudaMemcpyAsync(level, ld, bytes, cudaMemcpyDeviceToHost, s));
        LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return check_device_status(A, s);
} catch (...) {
    return lilac::api_failure();
}
