// Sliced ELL copies of a matrix (SELL-C-sigma with C = 32), built once per
// handle on first use (or for the tuner's trial) and kept with it, like the
// other invariants cached at create.  Two forms:
//
// SELL  Rows longer than the piece cap are cut into pieces of that many
//       nonzeros; rows and pieces ("lanes") are kept in row order when that
//       pads little, else sorted by length, longest first (stable); chunk c
//       holds lanes 32c .. 32c + 31, padded to the longest.  Built from the
//       host copy of row_ptr alone: the device scatters columns and values
//       into place.
//
// SLAB  The columns are cut into S slabs of W columns, W * 8 bytes at most
//       kSlabMaxBytes, S as small as that allows, and the rows into G = SMs / S
//       groups of about equal nonzero count.  For every (slab, group) pair,
//       the pieces of the group's rows (the row's nonzeros whose column lies
//       in the slab, in CSR order, 16-bit local columns) are sorted by length
//       and cut into chunks the same way, one CTA per pair; every row has a
//       (possibly empty) piece in every slab, so P[s][row] is always written.
//       Padding points at local column W, a zero kept after the slab of x in
//       shared memory.  A permutation (element -> CSR position, -1 for
//       padding) re-gathers the values after lilac_csr_update_values.
#include <algorithm>
#include <cstring>
#include <vector>

#include "launch.cuh"

namespace lilac {

namespace {

// Rows longer than this are cut into pieces: four times the mean row
// length rounded up to a power of two, 32 .. 4096.
int sell_piece_cap(const lilac_csr_s* A) {
    int cap = 32;
    while (cap < 4.0 * A->mean_row_len && cap < 4096) cap *= 2;
    return cap;
}

// Stable order of lanes by length, longest first (counting sort).
std::vector<int32_t> order_by_length(const std::vector<int32_t>& len, int maxlen) {
    std::vector<int64_t> start((size_t)maxlen + 2, 0);
    for (int32_t L : len) start[(size_t)(maxlen - L)]++;
    int64_t acc = 0;
    for (auto& c : start) {
        const int64_t t = c;
        c = acc;
        acc += t;
    }
    std::vector<int32_t> ord(len.size());
    for (size_t i = 0; i < len.size(); ++i) ord[(size_t)start[(size_t)(maxlen - len[i])]++] = (int32_t)i;
    return ord;
}

// Padded elements of the chunks of lanes taken in `ord` order (identity if empty).
int64_t padded_elems(const std::vector<int32_t>& len, const std::vector<int32_t>& ord) {
    const int64_t V = (int64_t)len.size();
    int64_t tot = 0;
    for (int64_t c = 0; c * 32 < V; ++c) {
        int32_t w = 0;
        for (int64_t i = c * 32; i < std::min(V, c * 32 + 32); ++i)
            w = std::max(w, len[(size_t)(ord.empty() ? i : ord[(size_t)i])]);
        tot += 32 * (int64_t)w;
    }
    return tot;
}

int slab_count(const lilac_csr_s* A, int* W) {
    const int64_t per = kSlabMaxBytes / 8;
    const int64_t S = A->ncols > 0 ? (A->ncols + per - 1) / per : 0;
    int64_t w = S > 0 ? (A->ncols + S - 1) / S : 0;
    w = (w + 7) & ~int64_t(7);
    *W = (int)w;
    return (int)S;
}

}  // namespace

// ---------------------------------------------------------------------------
// SELL

// Columns (unless `scol` is null) and values of every lane into place; one
// warp per chunk, lane l copies its row or piece with stride 32.
template <class T>
__global__ void sell_scatter_kernel(int nchunks, const int* __restrict__ cptr,
                                    const int* __restrict__ crow, const int4* __restrict__ splits,
                                    const int* __restrict__ piece_split, int cap,
                                    const int* __restrict__ row_ptr, const int* __restrict__ col,
                                    const T* __restrict__ val, int* __restrict__ scol,
                                    T* __restrict__ sval) {
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * (int64_t)blockDim.x) >> 5);
    for (int ch = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); ch < nchunks;
         ch += nwarps) {
        const int who = crow[(size_t)ch * 32 + lane];
        if (who == -1) continue;
        int src, len;
        if (who >= 0) {
            src = row_ptr[who];
            len = row_ptr[who + 1] - src;
        } else {
            const int p = -who - 2;
            const int4 sp = splits[piece_split[p]];
            const int re = row_ptr[sp.x + 1];
            src = row_ptr[sp.x] + (p - sp.y) * cap;
            len = min(cap, re - src);
        }
        const int64_t dst = (int64_t)cptr[ch] + lane;
        for (int k = 0; k < len; ++k) {
            if (scol) scol[dst + 32 * (int64_t)k] = col[src + k];
            sval[dst + 32 * (int64_t)k] = val[src + k];
        }
    }
}

template <class T>
static lilac_status sell_scatter(lilac_csr A, bool with_cols, cudaStream_t s) {
    if (A->sell_nchunks == 0) return LILAC_OK;
    sell_scatter_kernel<T><<<A->sm_count * 8, 256, 0, s>>>(
        A->sell_nchunks, A->sell_cptr.as<int>(), A->sell_crow.as<int>(), A->sell_splits.as<int4>(),
        A->sell_piece_split.as<int>(), A->sell_cap, A->row_ptr.as<int>(), A->col_ind.as<int>(),
        A->val.as<T>(), with_cols ? A->sell_col.as<int>() : nullptr, A->sell_val.as<T>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

static lilac_status build_sell(lilac_csr A, cudaStream_t s) {
    const int n = A->rows;
    const auto& rp = A->h_row_ptr;
    const int cap = sell_piece_cap(A);
    // lanes in row order: a row, or the pieces of a row longer than the cap
    std::vector<int32_t> who, len;
    who.reserve((size_t)n);
    len.reserve((size_t)n);
    std::vector<int4> splits;
    std::vector<int32_t> piece_split;
    for (int r = 0; r < n; ++r) {
        const int L = rp[r + 1] - rp[r];
        if (L <= cap) {
            who.push_back(r);
            len.push_back(L);
            continue;
        }
        const int lid = (int)splits.size();
        const int np = (L + cap - 1) / cap;
        const int first = (int)piece_split.size();
        splits.push_back(make_int4(r, first, np, 0));
        for (int j = 0; j < np; ++j) {
            piece_split.push_back(lid);
            who.push_back(-(2 + first + j));
            len.push_back(std::min(cap, L - j * cap));
        }
    }
    const int64_t V = (int64_t)who.size();
    if (V >= (int64_t(1) << 31) / 32) return LILAC_OK;  // too many lanes: not built
    // row order when it pads little (keeps the epilogue and x accesses
    // local), else sorted by length
    std::vector<int32_t> ord;
    int64_t elems = padded_elems(len, ord);
    int sigma = 1;
    if ((double)elems > 1.1 * (double)A->nnz + 32.0 * (double)((V + 31) / 32)) {
        std::vector<int32_t> sorted = order_by_length(len, cap);
        const int64_t e2 = padded_elems(len, sorted);
        if (e2 < elems) {
            ord.swap(sorted);
            elems = e2;
            sigma = 0;  // whole matrix
        }
    }
    // not worth a copy when padding adds more than half, or offsets overflow
    if ((double)elems > 1.5 * (double)A->nnz + 64.0 * (double)((V + 31) / 32) ||
        elems >= (int64_t(1) << 31) - 64)
        return LILAC_OK;
    const int nch = (int)((V + 31) / 32);
    std::vector<int32_t> cptr((size_t)nch + 1), crow((size_t)nch * 32, -1);
    cptr[0] = 0;
    for (int c = 0; c < nch; ++c) {
        int32_t w = 0;
        for (int l = 0; l < 32; ++l) {
            const int64_t i = (int64_t)c * 32 + l;
            if (i >= V) break;
            const int32_t lane_i = ord.empty() ? (int32_t)i : ord[(size_t)i];
            crow[(size_t)i] = who[(size_t)lane_i];
            w = std::max(w, len[(size_t)lane_i]);
        }
        cptr[(size_t)c + 1] = cptr[(size_t)c] + 32 * w;
    }
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    const size_t epad = (size_t)elems + 64;
    const size_t nsplit = splits.size(), npieces = piece_split.size();
    LILAC_TRY(A->ws_alloc(A->sell_cptr, sizeof(int32_t) * cptr.size()));
    LILAC_TRY(A->ws_alloc(A->sell_crow, sizeof(int32_t) * crow.size()));
    LILAC_TRY(A->ws_alloc(A->sell_col, sizeof(int32_t) * epad));
    LILAC_TRY(A->ws_alloc(A->sell_val, vsz * epad));
    LILAC_TRY(A->ws_alloc(A->sell_splits, sizeof(int4) * std::max<size_t>(1, nsplit)));
    LILAC_TRY(A->ws_alloc(A->sell_piece_split, sizeof(int32_t) * std::max<size_t>(1, npieces)));
    LILAC_TRY(A->ws_alloc(A->sell_part, sizeof(double) * std::max<size_t>(1, npieces)));
    LILAC_TRY(A->ws_alloc(A->sell_red, sizeof(double) * kMaxRed * std::max<size_t>(1, nsplit)));
    LILAC_TRY(A->ws_alloc(A->sell_cnt, sizeof(unsigned) * std::max<size_t>(1, nsplit)));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->sell_col.p, 0xff, A->sell_col.bytes, s));  // -1: padding
    LILAC_CUDA_TRY(cudaMemsetAsync(A->sell_val.p, 0, A->sell_val.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->sell_part.p, 0, A->sell_part.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->sell_red.p, 0, A->sell_red.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->sell_cnt.p, 0, A->sell_cnt.bytes, s));
    auto up = [&](lilac::DevBuf& d, const void* h, size_t bytes) -> lilac_status {
        if (bytes) LILAC_CUDA_TRY(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, s));
        return LILAC_OK;
    };
    LILAC_TRY(up(A->sell_cptr, cptr.data(), sizeof(int32_t) * cptr.size()));
    LILAC_TRY(up(A->sell_crow, crow.data(), sizeof(int32_t) * crow.size()));
    LILAC_TRY(up(A->sell_splits, splits.data(), sizeof(int4) * nsplit));
    LILAC_TRY(up(A->sell_piece_split, piece_split.data(), sizeof(int32_t) * npieces));
    A->sell_nchunks = nch;
    A->sell_nsplit = (int)nsplit;
    A->sell_npieces = (int)npieces;
    A->sell_cap = cap;
    A->sell_sigma = sigma;
    A->sell_elems = elems;
    // sorted rows: an epilogue that reads per-row data would scatter; where
    // rows are many and short, its reductions run as a second, row-order pass
    A->sell_two_pass = sigma == 0 && n >= (1 << 16) && A->mean_row_len < 64.0;
    LILAC_TRY(A->dtype == LILAC_F64 ? sell_scatter<double>(A, true, s) : sell_scatter<float>(A, true, s));
    // the host vectors above must outlive the copies
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->sell_built = nch > 0;
    return LILAC_OK;
}

lilac_status sell_refresh_values(lilac_csr A, cudaStream_t s) {
    if (!A->sell_built) return LILAC_OK;
    return A->dtype == LILAC_F64 ? sell_scatter<double>(A, false, s) : sell_scatter<float>(A, false, s);
}

lilac_status sell_zero_counters(lilac_csr A, cudaStream_t s) {
    if (A->sell_cnt.p) LILAC_CUDA_TRY(cudaMemsetAsync(A->sell_cnt.p, 0, A->sell_cnt.bytes, s));
    return LILAC_OK;
}

void sell_release(lilac_csr A) {
    lilac::DevBuf* b[] = {&A->sell_cptr,  &A->sell_crow,        &A->sell_col,
                          &A->sell_val,   &A->sell_splits,      &A->sell_piece_split,
                          &A->sell_part,  &A->sell_red,         &A->sell_cnt};
    for (auto* d : b) d->release();
    A->sell_nchunks = A->sell_nsplit = A->sell_npieces = A->sell_cap = A->sell_sigma = 0;
    A->sell_elems = 0;
    A->sell_built = false;
    A->sell_two_pass = false;
}

lilac_status ensure_sell(lilac_csr A, cudaStream_t s) {
    if (A->sell_built || A->rows == 0 || A->nnz == 0) return LILAC_OK;
    return build_sell(A, s);
}

// ---------------------------------------------------------------------------
// SLAB

// Worth building when x is too large for L1 yet a handful of slabs holds it,
// each CTA's share of the nonzeros is large, and rows are long enough per
// slab to amortise the per-row work.
bool slab_worthwhile(const lilac_csr_s* A) {
    if (A->nnz == 0 || A->rows == 0 || A->ncols == 0) return false;
    int W = 0;
    const int S = slab_count(A, &W);
    return (int64_t)A->ncols * 8 > (128 << 10) && S <= 8 && S <= A->sm_count &&
           A->mean_row_len >= 8.0 * S && A->nnz >= (int64_t)A->sm_count * 4096;
}

template <class T>
__global__ void slab_regather_kernel(int64_t elems, const int* __restrict__ perm,
                                     const T* __restrict__ val, T* __restrict__ sval) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < elems;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = perm[q];
        sval[q] = k >= 0 ? val[k] : T(0);
    }
}

template <class T>
static lilac_status regather(lilac_csr A, int64_t elems, cudaStream_t s) {
    if (elems == 0) return LILAC_OK;
    slab_regather_kernel<T><<<A->sm_count * 8, 256, 0, s>>>(elems, A->slab_perm.as<int>(),
                                                             A->val.as<T>(), A->slab_val.as<T>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

static lilac_status build_slab(lilac_csr A, cudaStream_t s) {
    const int n = A->rows;
    const int64_t nnz = A->nnz;
    int W = 0;
    const int S = slab_count(A, &W);
    const auto& rp = A->h_row_ptr;
    std::vector<int32_t> col((size_t)nnz);
    LILAC_CUDA_TRY(cudaMemcpyAsync(col.data(), A->col_ind.p, sizeof(int32_t) * (size_t)nnz,
                                   cudaMemcpyDeviceToHost, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    // piece length of every (slab, row)
    std::vector<int32_t> cnt((size_t)S * (size_t)n, 0);
    for (int r = 0; r < n; ++r)
        for (int k = rp[r]; k < rp[r + 1]; ++k) cnt[(size_t)(col[(size_t)k] / W) * n + r]++;
    // row groups of about equal nonzero count, one CTA per (slab, group)
    const int G0 = std::max(1, A->sm_count / std::max(1, S));
    std::vector<int2> groups;
    {
        int r = 0;
        for (int g = 0; g < G0 && r < n; ++g) {
            const int ra = r;
            if (g == G0 - 1) {
                r = n;
            } else {
                const int64_t target = nnz * (g + 1) / G0;
                while (r < n && rp[r + 1] <= target) ++r;
                if (r == ra) ++r;
            }
            groups.push_back(make_int2(ra, r));
        }
    }
    const int G = (int)groups.size();
    // sliced ELL chunks of each (slab, group): the group's rows sorted by piece
    // length, longest first
    std::vector<int32_t> cptr(1, 0), crow;
    std::vector<int4> ctas;
    std::vector<int64_t> base((size_t)S * (size_t)n);  // first element of each piece
    int64_t elems = 0;
    for (int sl = 0; sl < S; ++sl) {
        for (int g = 0; g < G; ++g) {
            const int r0 = groups[(size_t)g].x, r1 = groups[(size_t)g].y;
            const std::vector<int32_t> len(cnt.begin() + (size_t)sl * n + r0,
                                           cnt.begin() + (size_t)sl * n + r1);
            const int maxlen = *std::max_element(len.begin(), len.end());
            const std::vector<int32_t> ord = order_by_length(len, maxlen);
            const int nr = r1 - r0;
            const int first = (int)cptr.size() - 1;
            for (int c = 0; c * 32 < nr; ++c) {
                int32_t w = 0;
                for (int l = 0; l < 32; ++l) {
                    const int i = c * 32 + l;
                    if (i >= nr) {
                        crow.push_back(-1);
                        continue;
                    }
                    const int r = r0 + ord[(size_t)i];
                    crow.push_back(r);
                    base[(size_t)sl * n + r] = elems + l;
                    w = std::max(w, len[(size_t)ord[(size_t)i]]);
                }
                elems += 32 * (int64_t)w;
                if (elems >= (int64_t(1) << 31) - 64) return LILAC_OK;  // offsets overflow: not built
                cptr.push_back((int32_t)elems);
            }
            ctas.push_back(make_int4(sl, first, (int)cptr.size() - 1, g));
        }
    }
    // padding of more than a quarter: not worth the copy (STAGED runs)
    if ((double)elems > 1.25 * (double)nnz + 32.0 * (double)crow.size()) return LILAC_OK;
    // CG form: the chunks of slab s (all its groups, contiguous) cut into G
    // runs of about equal padded element counts, one CTA each
    std::vector<int4> ranges;
    for (int sl = 0; sl < S; ++sl) {
        const int cb = ctas[(size_t)sl * G].y, ce = ctas[(size_t)sl * G + G - 1].z;
        const int64_t eb = cptr[(size_t)cb], ee = cptr[(size_t)ce];
        int cur = cb;
        for (int j = 0; j < G; ++j) {
            int nxt = ce;
            if (j < G - 1) {
                const int64_t target = eb + (ee - eb) * (j + 1) / G;
                nxt = cur;
                while (nxt < ce && cptr[(size_t)nxt + 1] <= target) ++nxt;
            }
            ranges.push_back(make_int4(sl, cur, nxt, 0));
            cur = nxt;
        }
    }
    std::vector<int32_t> perm((size_t)elems, -1);
    std::vector<uint16_t> c16((size_t)elems, (uint16_t)W);
    {
        std::vector<int32_t> fill((size_t)S);
        for (int r = 0; r < n; ++r) {
            std::fill(fill.begin(), fill.end(), 0);
            for (int k = rp[r]; k < rp[r + 1]; ++k) {
                const int c = col[(size_t)k];
                const int sl = c / W;
                const int64_t q = base[(size_t)sl * n + r] + 32 * (int64_t)fill[(size_t)sl]++;
                perm[(size_t)q] = k;
                c16[(size_t)q] = (uint16_t)(c - sl * W);
            }
        }
    }
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    const size_t epad = (size_t)elems + 64;
    LILAC_TRY(A->ws_alloc(A->slab_cptr, sizeof(int32_t) * cptr.size()));
    LILAC_TRY(A->ws_alloc(A->slab_crow, sizeof(int32_t) * crow.size()));
    LILAC_TRY(A->ws_alloc(A->slab_col, sizeof(uint16_t) * epad));
    LILAC_TRY(A->ws_alloc(A->slab_val, vsz * epad));
    LILAC_TRY(A->ws_alloc(A->slab_perm, sizeof(int32_t) * std::max<size_t>(1, (size_t)elems)));
    LILAC_TRY(A->ws_alloc(A->slab_ctas, sizeof(int4) * ctas.size()));
    LILAC_TRY(A->ws_alloc(A->slab_groups, sizeof(int2) * groups.size()));
    LILAC_TRY(A->ws_alloc(A->slab_gcnt, sizeof(unsigned) * groups.size()));
    LILAC_TRY(A->ws_alloc(A->slab_P, sizeof(double) * (size_t)S * (size_t)std::max(1, n)));
    LILAC_TRY(A->ws_alloc(A->slab_ranges, sizeof(int4) * ranges.size()));
    LILAC_TRY(A->ws_alloc(A->slab_pq, sizeof(double) * ranges.size()));
    // the CG form keeps its chunks' p[row] * piece in shared memory after the
    // slab when the longest run fits (kSlabCgSmemBytes in all), else in T
    int maxch = 0;
    for (const int4& rg : ranges) maxch = std::max(maxch, rg.z - rg.y);
    const size_t slab_bytes = sizeof(double) * (((size_t)W + 2) & ~size_t(1));
    const size_t t_bytes = sizeof(double) * 32 * (size_t)maxch;
    A->slab_tsm = slab_bytes + t_bytes <= kSlabCgSmemBytes ? 1 : 0;
    A->slab_cg_smem = A->slab_tsm ? slab_bytes + t_bytes : slab_bytes;
    if (!A->slab_tsm) LILAC_TRY(A->ws_alloc(A->slab_T, sizeof(double) * crow.size()));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_val.p, 0, A->slab_val.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_gcnt.p, 0, A->slab_gcnt.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->slab_P.p, 0, A->slab_P.bytes, s));
    auto up = [&](lilac::DevBuf& d, const void* h, size_t bytes) -> lilac_status {
        if (bytes) LILAC_CUDA_TRY(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, s));
        return LILAC_OK;
    };
    LILAC_TRY(up(A->slab_cptr, cptr.data(), sizeof(int32_t) * cptr.size()));
    LILAC_TRY(up(A->slab_crow, crow.data(), sizeof(int32_t) * crow.size()));
    LILAC_TRY(up(A->slab_col, c16.data(), sizeof(uint16_t) * c16.size()));
    LILAC_TRY(up(A->slab_perm, perm.data(), sizeof(int32_t) * perm.size()));
    LILAC_TRY(up(A->slab_ctas, ctas.data(), sizeof(int4) * ctas.size()));
    LILAC_TRY(up(A->slab_groups, groups.data(), sizeof(int2) * groups.size()));
    LILAC_TRY(up(A->slab_ranges, ranges.data(), sizeof(int4) * ranges.size()));
    LILAC_TRY(A->dtype == LILAC_F64 ? regather<double>(A, elems, s) : regather<float>(A, elems, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->slab_S = S;
    A->slab_W = W;
    A->slab_G = G;
    A->slab_grid = (int)ctas.size();
    A->slab_elems = elems;
    A->slab_built = !ctas.empty();
    return LILAC_OK;
}

// After new values were uploaded: rebuild the regrouped values on the device.
lilac_status slab_refresh_values(lilac_csr A, cudaStream_t s) {
    if (!A->slab_built) return LILAC_OK;
    return A->dtype == LILAC_F64 ? regather<double>(A, A->slab_elems, s)
                                 : regather<float>(A, A->slab_elems, s);
}

void slab_release(lilac_csr A) {
    lilac::DevBuf* b[] = {&A->slab_cptr,  &A->slab_crow,   &A->slab_col,  &A->slab_val,
                          &A->slab_perm,  &A->slab_ctas,   &A->slab_groups, &A->slab_gcnt,
                          &A->slab_P,     &A->slab_ranges, &A->slab_T, &A->slab_pq};
    for (auto* d : b) d->release();
    A->slab_S = A->slab_W = A->slab_grid = A->slab_G = 0;
    A->slab_tsm = 0;
    A->slab_cg_smem = 0;
    A->slab_elems = 0;
    A->slab_built = false;
}

lilac_status ensure_slab(lilac_csr A, cudaStream_t s) {
    if (A->slab_built) return LILAC_OK;
    int W = 0;
    const int S = slab_count(A, &W);
    if (A->nnz == 0 || S == 0) return LILAC_OK;  // nothing to regroup: STAGED runs
    // too many slabs for the layout: not built, STAGED runs
    if (S > 64 || (int64_t)S * ((int64_t)A->rows + 32) >= (int64_t(1) << 31) - 64) return LILAC_OK;
    return build_slab(A, s);
}

}  // namespace lilac
