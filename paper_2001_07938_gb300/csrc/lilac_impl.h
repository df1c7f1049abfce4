// Internal host-side definitions: the handle, error plumbing, device
// buffers, and the SpMV launch dispatcher shared by the entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lilac.h"
#include "ops.cuh"

namespace lilac {

// Tile shape of the STAGED kernel: at most kTileNnz nonzeros and kTileRows
// rows per tile, kStagedThreads threads per CTA (overridable at build time).
#ifndef LILAC_STAGED_THREADS
#define LILAC_STAGED_THREADS 256
#endif
#ifndef LILAC_TILE_NNZ
#define LILAC_TILE_NNZ 2048
#endif
#ifndef LILAC_TILE_ROWS
#define LILAC_TILE_ROWS 1024
#endif
constexpr int kStagedThreads = LILAC_STAGED_THREADS;
constexpr int kTileNnz = LILAC_TILE_NNZ;
constexpr int kTileRows = LILAC_TILE_ROWS;
constexpr int kRowsThreads = 256;
// SLAB kernel shape: one CTA of 1024 threads per SM with a slab of x of at
// most kSlabMaxBytes (x elements counted as 8 bytes) in shared memory.
constexpr int kSlabThreads = 1024;
constexpr int kSlabMaxBytes = 192 * 1024;
// Shared memory of the CG form of SLAB at most: the slab plus its chunks'
// p.q terms when they fit.
constexpr size_t kSlabCgSmemBytes = 224 * 1024;
// MERGE kernel shape: 256 threads, sub-tiles of 2048 path items (8 per
// thread); overridable at build time.
#ifndef LILAC_MERGE_THREADS
#define LILAC_MERGE_THREADS 256
#endif
#ifndef LILAC_MERGE_ITEMS
#define LILAC_MERGE_ITEMS 2048
#endif
constexpr int kMergeThreads = LILAC_MERGE_THREADS;
constexpr int kMergeItems = LILAC_MERGE_ITEMS;
constexpr int kMaxCtas = 8192;  // bound of the per-CTA partial-sum buffer

void set_last_error(const std::string& msg);
lilac_status api_failure() noexcept;

#define LILAC_CUDA_TRY(...)                                                                   \
    do {                                                                                      \
        cudaError_t _e = (__VA_ARGS__);                                                       \
        if (_e != cudaSuccess) {                                                              \
            ::lilac::set_last_error(std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(_e)); \
            return _e == cudaErrorMemoryAllocation ? LILAC_ERR_OOM : LILAC_ERR_CUDA;          \
        }                                                                                     \
    } while (0)

#define LILAC_TRY(...)                        \
    do {                                      \
        lilac_status _s = (__VA_ARGS__);      \
        if (_s != LILAC_OK) return _s;        \
    } while (0)

// Device allocation owned by a handle.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    lilac_status alloc(size_t n);
    void release();
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

struct CgWork {
    int n = 0;
    bool f32 = false;
    DevBuf r, p, q, state;  // vectors of the handle's CG precision; state = CgState
};

struct GraphKey {
    int kind;
    const void* a;
    const void* b;
    int iters;
    uint64_t extra;
    int variant;
    int vwidth;
    uint64_t gen;  // workspace generation of the handle at capture time
    bool operator<(const GraphKey& o) const {
        return std::tie(kind, a, b, iters, extra, variant, vwidth, gen) <
               std::tie(o.kind, o.a, o.b, o.iters, o.extra, o.variant, o.vwidth, o.gen);
    }
};

}  // namespace lilac

struct lilac_csr_s {
    int device = 0;
    int sm_count = 0;
    int32_t rows = 0, ncols = 0;
    int64_t nnz = 0;
    lilac_dtype dtype = LILAC_F64;
    // matrix (padded so that 16-byte-rounded bulk copies stay inside)
    lilac::DevBuf row_ptr, col_ind, val;
    lilac::DevBuf val32;  // FP32 copy of FP64 values, built on first mixed-precision use
    bool val32_valid = false;
    // row statistics (the invariants cached at create)
    int32_t max_row_len = 0, empty_rows = 0;
    double mean_row_len = 0.0, std_row_len = 0.0;
    // kernel choice, and the timed tuner's trial {variant, width, ms per call}
    int variant = LILAC_VARIANT_STAGED;
    int vwidth = 32;
    std::vector<std::tuple<int, int, float>> tune_table;
    // STAGED schedule
    lilac::DevBuf tiles, longs;
    int ntiles = 0, nlong = 0, nlong_chunks = 0;
    // SLAB copy (built on first use): sliced ELL chunks of the row pieces of
    // every (slab, row group) pair (chunk offsets, lane rows, 16-bit local
    // columns, values), the CSR index of each element (-1: padding; value
    // updates), CTA ranges {slab, first chunk, end chunk, group}, the groups'
    // rows, their arrival counters, and the partial sums P (S x rows)
    lilac::DevBuf slab_cptr, slab_crow, slab_col, slab_val, slab_perm, slab_ctas, slab_groups,
        slab_gcnt, slab_P;
    // CG form of SLAB: per-CTA runs of a slab's chunks with equal element
    // counts, one p[row] * piece per chunk lane (used when they do not fit in
    // shared memory: slab_tsm == 0), and the per-CTA p.q sums
    lilac::DevBuf slab_ranges, slab_T, slab_pq;
    int slab_tsm = 0;
    size_t slab_cg_smem = 0;
    int slab_S = 0, slab_W = 0, slab_grid = 0, slab_G = 0;
    int64_t slab_elems = 0;
    bool slab_built = false;
    // SELL copy (built on first use): chunk offsets, lane rows / pieces,
    // columns (-1: padding), values, split rows {row, first piece, pieces, -},
    // piece -> split row, and the split rows' piece sums, epilogue sums and
    // arrival counters
    lilac::DevBuf sell_cptr, sell_crow, sell_col, sell_val, sell_splits, sell_piece_split,
        sell_part, sell_red, sell_cnt;
    int sell_nchunks = 0, sell_nsplit = 0, sell_npieces = 0, sell_cap = 0, sell_sigma = 0;
    int64_t sell_elems = 0;
    bool sell_built = false;
    bool sell_two_pass = false;  // sorted rows, many of them: reductions in a row-order pass
    // HUB copies (built on first use; lilac_hub.cu): the hub columns and their
    // gathered x, the hot part (chunk offsets, lane rows / sub-pieces, 16-bit
    // slab-local columns, values, CSR index per element, CTA runs, slab
    // partials P, long pieces' splits with their sums and counters), and
    // the cold part as a sliced ELL copy (chunk offsets, lane rows / pieces,
    // columns, values, CSR index per element, split rows and their scratch,
    // per lane the mask of slabs in which its row has a piece)
    lilac::DevBuf hub_cols, hub_xhot, hub_cptr, hub_crow, hub_col, hub_val, hub_perm, hub_ranges,
        hub_P, hub_splits, hub_sub_split, hub_part, hub_cnt;
    lilac::DevBuf hubc_cptr, hubc_crow, hubc_col, hubc_val, hubc_perm, hubc_splits,
        hubc_piece_split, hubc_part, hubc_red, hubc_cnt, hubc_mask;
    int hub_H = 0, hub_S = 0, hub_W = 0, hub_grid = 0, hub_pstride = 0;
    int hubc_nchunks = 0, hubc_nsplit = 0, hubc_npieces = 0;
    int64_t hub_elems = 0, hubc_elems = 0;
    double hub_share = 0.0;
    bool hub_built = false;
    bool hub_two_pass = false;  // many short rows: reductions in a row-order pass
    // JDS copy (built on first use): slot -> row, row -> slot, slot lengths,
    // jagged diagonal offsets, columns and values in JDS order
    lilac::DevBuf jds_slot_row, jds_row_slot, jds_len, jds_ptr, jds_col, jds_val;
    int jds_njd = 0;
    bool jds_built = false;
    // MERGE partition (computed at create): start of each CTA's path range
    lilac::DevBuf merge_coords, merge_carries;
    int merge_grid = 0;
    int64_t merge_per_cta = 0;
    // scratch
    lilac::DevBuf partials, long_part, long_red, long_cnt, ticket, status;
    // host-pointer staging (marshaling of x / y for LILAC_MEM_HOST calls)
    lilac::DevBuf stage_x, stage_y;
    // solvers
    lilac::CgWork cg64, cg32;
    lilac::DevBuf cg_outer_state, cg_outer_r, ir_x, ir_b;  // mixed precision outer loop
    // fused CG step after the SLAB CG form: grid barrier counters [2] (zero
    // between launches), then one r.r partial per CTA
    lilac::DevBuf cg_step;
    lilac::DevBuf pr_y, pr_state, pr_l1, pr_has_out;
    bool pr_has_out_valid = false;
    // BFS: row index of every nonzero (built on first use), state, staged levels
    lilac::DevBuf bfs_row, bfs_state, bfs_level;
    // SpMM: staging / transposition scratch
    lilac::DevBuf spmm_buf;
    cudaStream_t capture_stream = nullptr;
    std::map<lilac::GraphKey, cudaGraphExec_t> graphs;
    std::vector<cudaEvent_t> prof_events;  // pairs around timed SpMV launches
    bool profiling = false;                // lilac_csr_profile switch
    double prof_ms_acc = 0.0;
    int64_t prof_launches_acc = 0;
    // host copies
    std::vector<int32_t> h_row_ptr;
    int64_t h2d_bytes = 0;
    bool sticky_error = false;
    uint64_t ws_gen = 0;  // bumped whenever a buffer a captured graph may use is reallocated

    // (Re)allocate a workspace buffer; cached graphs that used the old one
    // stop matching.
    lilac_status ws_alloc(lilac::DevBuf& b, size_t bytes) {
        ++ws_gen;
        return b.alloc(bytes);
    }

    lilac::Scratch scratch() const;
    int64_t device_bytes() const;
};

namespace lilac {

// Switch to the handle's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

lilac_status check_handle(lilac_csr A);
lilac_status make_val32(lilac_csr A, cudaStream_t stream);
lilac_status ensure_slab(lilac_csr A, cudaStream_t stream);
lilac_status ensure_jds(lilac_csr A, cudaStream_t stream);
lilac_status jds_refresh_values(lilac_csr A, cudaStream_t stream);
void jds_release(lilac_csr A);
lilac_status slab_refresh_values(lilac_csr A, cudaStream_t stream);
void slab_release(lilac_csr A);
bool slab_worthwhile(const lilac_csr_s* A);
lilac_status ensure_sell(lilac_csr A, cudaStream_t stream);
// One CG solve on caller-held device memory with the handle's tuned kernels
// (lilac_cg.cu; the request server's lane for large matrices).  prec 0: FP64
// CG; prec 2: FP32 CG with FP64 reliable updates (delta: the replacement
// threshold).  Bytes of the caller's workspace, its layout, preparation
// (before any capture), the start (x = 0) and nit iterations as a cached graph.
struct SoloCg {
    CgWork W;  // views into the caller's workspace
    float* d = nullptr;
    double* r64 = nullptr;
    int prec = 0;
};
size_t solo_cg_bytes(const lilac_csr_s* A, int prec);
void solo_cg_bind(const lilac_csr_s* A, int prec, void* ws, SoloCg& c);
lilac_status solo_cg_prepare(lilac_csr A, int prec, cudaStream_t s);
lilac_status solo_cg_start(lilac_csr A, SoloCg& c, const double* b, double* x, double rtol,
                           int max_iter, double delta, cudaStream_t s);
lilac_status solo_cg_iters(lilac_csr A, SoloCg& c, const double* b, double* x, int nit,
                           cudaStream_t s);
lilac_status spmm_vectors_device(lilac_csr A, int k, const double* Xv, double* Yv, double* scratch,
                                 cudaStream_t s);
bool hub_worthwhile(const lilac_csr_s* A);
lilac_status ensure_hub(lilac_csr A, cudaStream_t stream);
lilac_status hub_refresh_values(lilac_csr A, cudaStream_t stream);
lilac_status hub_zero_counters(lilac_csr A, cudaStream_t stream);
void hub_release(lilac_csr A);
lilac_status sell_refresh_values(lilac_csr A, cudaStream_t stream);
void sell_release(lilac_csr A);
lilac_status sell_zero_counters(lilac_csr A, cudaStream_t stream);
lilac_status check_device_status(lilac_csr A, cudaStream_t stream);
// Event pairs for timing SpMV launches (pair i = events 2i, 2i+1).
lilac_status ensure_prof_events(lilac_csr A, int pairs);
// Sum the durations of the first `pairs` pairs (their work must be complete).
lilac_status collect_prof_events(lilac_csr A, int pairs, double* ms, int* launches);
int vec_grid(const lilac_csr_s* A, int64_t n);

}  // namespace lilac
