// HUB copies of a matrix (the HUB kernels of spmv_kernels.cuh), built once
// per handle on first use or for the tuner's trial, like the SELL and SLAB
// copies, and kept only if they win:
//
//   hub columns  the H most frequent columns (ties: the lower column first),
//                in column order: slot h holds column hub_cols[h]; slab h / W
//                of at most W = 192 KB of x, S <= 5 slabs (a slab is added
//                while it covers at least 3% more of the nonzeros)
//   hot part     per slab, the piece of every row that has one (its nonzeros
//                in the slab's hub columns, in CSR order) as one lane, or as
//                sub-pieces of at most kHubPieceCap, one lane each; lanes
//                sorted by piece length, longest first (stable), in chunks of
//                32 padded to the longest; 16-bit slab-local columns (padding:
//                W, a zero); CTA runs of about equal work (elements, plus
//                kHubChunkCost per chunk for its fixed latency)
//   cold part    the other nonzeros of every row as a sliced ELL copy laid
//                out like SELL's (lanes sorted by length, rows longer than
//                the piece cap cut into pieces), original columns (padding
//                -1), and per lane the mask of slabs the row has pieces in
//
// Both parts keep each element's CSR index (-1: padding) so that value
// updates are gathered again on the device.  Not built when the hub columns
// hold less than kHubMinShare of the nonzeros, or less than twice their share
// of the columns (no concentration: uniform columns).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "launch.cuh"

namespace lilac {

namespace {

// At most 8 slabs (the cold copy's per-lane slab mask is one byte).
#ifndef LILAC_HUB_MAX_SLABS
#define LILAC_HUB_MAX_SLABS 5
#endif
#ifndef LILAC_HUB_SLAB_GAIN
#define LILAC_HUB_SLAB_GAIN 0.03
#endif
constexpr int kHubMaxSlabs = LILAC_HUB_MAX_SLABS;
static_assert(kHubMaxSlabs >= 1 && kHubMaxSlabs <= 8, "the slab mask is one byte");
constexpr double kHubMinShare = 0.4;
constexpr double kHubSlabGain = LILAC_HUB_SLAB_GAIN;
constexpr int64_t kHubMinXBytes = int64_t(1) << 20;
constexpr int64_t kHubChunkCost = 256;
constexpr int kHubPieceCap = 1024;  // hot elements per lane at most

// x values per slab: 192 KB (FP32: 49,152, FP64: 24,576), below the 16-bit
// local column range with one padding slot.
int hub_slab_width(size_t vsz) { return (int)((size_t)kSlabMaxBytes / vsz); }

// Stable order of lanes by length, longest first (counting sort).
std::vector<int32_t> by_length(const std::vector<int32_t>& len, int maxlen) {
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

template <class T>
__global__ void hub_regather_kernel(int64_t elems, const int* __restrict__ perm,
                                    const T* __restrict__ val, T* __restrict__ out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < elems;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int k = perm[q];
        out[q] = k >= 0 ? val[k] : T(0);
    }
}

template <class T>
lilac_status hub_regather(lilac_csr A, cudaStream_t s) {
    if (A->hub_elems > 0)
        hub_regather_kernel<T><<<A->sm_count * 8, 256, 0, s>>>(
            A->hub_elems, A->hub_perm.as<int>(), A->val.as<T>(), A->hub_val.as<T>());
    if (A->hubc_elems > 0)
        hub_regather_kernel<T><<<A->sm_count * 8, 256, 0, s>>>(
            A->hubc_elems, A->hubc_perm.as<int>(), A->val.as<T>(), A->hubc_val.as<T>());
    LILAC_CUDA_TRY(cudaGetLastError());
    return LILAC_OK;
}

}  // namespace

bool hub_worthwhile(const lilac_csr_s* A) {
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    return A->rows > 0 && A->nnz >= (int64_t)A->sm_count * 4096 &&
           (int64_t)A->ncols * (int64_t)vsz > kHubMinXBytes && A->ncols > hub_slab_width(vsz);
}

static lilac_status build_hub(lilac_csr A, cudaStream_t s) {
    const int n = A->rows, ncols = A->ncols;
    const int64_t nnz = A->nnz;
    const size_t vsz = A->dtype == LILAC_F64 ? 8 : 4;
    const int W = hub_slab_width(vsz);
    const auto& rp = A->h_row_ptr;
    std::vector<int32_t> col((size_t)nnz);
    LILAC_CUDA_TRY(cudaMemcpyAsync(col.data(), A->col_ind.p, sizeof(int32_t) * (size_t)nnz,
                                   cudaMemcpyDeviceToHost, s));
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int64_t> cnt((size_t)ncols, 0);
    for (int64_t k = 0; k < nnz; ++k) cnt[(size_t)col[(size_t)k]]++;
    // the most frequent columns and the share the first 1 .. S slabs of them hold
    const int64_t hmax = std::min<int64_t>(ncols, (int64_t)kHubMaxSlabs * W);
    std::vector<int32_t> idx((size_t)ncols);
    std::iota(idx.begin(), idx.end(), 0);
    std::partial_sort(idx.begin(), idx.begin() + hmax, idx.end(), [&](int32_t a, int32_t b) {
        return cnt[(size_t)a] != cnt[(size_t)b] ? cnt[(size_t)a] > cnt[(size_t)b] : a < b;
    });
    std::vector<double> share(kHubMaxSlabs + 1, 0.0);
    {
        int64_t acc = 0, h = 0;
        for (int sl = 1; sl <= kHubMaxSlabs; ++sl) {
            const int64_t end = std::min<int64_t>(hmax, (int64_t)sl * W);
            for (; h < end; ++h) acc += cnt[(size_t)idx[(size_t)h]];
            share[sl] = (double)acc / (double)nnz;
        }
    }
    int S = 1;
    while (S < kHubMaxSlabs && (int64_t)S * W < ncols && share[S + 1] - share[S] >= kHubSlabGain) ++S;
    const int H = (int)std::min<int64_t>(ncols, (int64_t)S * W);
    if (share[S] < kHubMinShare || share[S] < 2.0 * H / ncols) return LILAC_OK;  // STAGED runs
    S = (H + W - 1) / W;
    std::vector<int32_t> hot(idx.begin(), idx.begin() + H);
    std::sort(hot.begin(), hot.end());
    std::vector<int32_t> slot((size_t)ncols, -1);
    for (int h = 0; h < H; ++h) slot[(size_t)hot[(size_t)h]] = h;
    idx.clear();
    idx.shrink_to_fit();
    // piece lengths per (slab, row) and cold lengths per row
    std::vector<int32_t> plen((size_t)S * n, 0), clen((size_t)n, 0);
    for (int r = 0; r < n; ++r)
        for (int k = rp[r]; k < rp[r + 1]; ++k) {
            const int h = slot[(size_t)col[(size_t)k]];
            if (h >= 0)
                plen[(size_t)(h / W) * n + r]++;
            else
                clen[(size_t)r]++;
        }
    // the slabs a row has pieces in
    auto row_mask = [&](int r) {
        int m = 0;
        for (int sl = 0; sl < S; ++sl)
            if (plen[(size_t)sl * n + r] > 0) m |= 1 << sl;
        return m;
    };
    // hot part: per slab, lanes are the rows with a piece, or sub-pieces of at
    // most kHubPieceCap of a longer piece (split), sorted by length
    const int G = std::max(1, A->sm_count / S);
    std::vector<int32_t> hcptr(1, 0), hcrow;
    std::vector<int4> ranges, hsplits;
    std::vector<int32_t> hsub_split, hsplit_of((size_t)S * n, -1);
    std::vector<int64_t> hbase((size_t)S * n, -1), subbase;
    int64_t helems = 0;
    for (int sl = 0; sl < S; ++sl) {
        std::vector<int32_t> lwho, llen;
        for (int r = 0; r < n; ++r) {
            const int L = plen[(size_t)sl * n + r];
            if (L == 0) continue;
            if (L <= kHubPieceCap) {
                lwho.push_back(r);
                llen.push_back(L);
                continue;
            }
            const int lid = (int)hsplits.size();
            const int ns = (L + kHubPieceCap - 1) / kHubPieceCap;
            const int firsts = (int)hsub_split.size();
            hsplits.push_back(make_int4(r, firsts, ns, sl));
            hsplit_of[(size_t)sl * n + r] = lid;
            for (int q = 0; q < ns; ++q) {
                hsub_split.push_back(lid);
                lwho.push_back(-(2 + firsts + q));
                llen.push_back(std::min(kHubPieceCap, L - q * kHubPieceCap));
            }
        }
        subbase.resize(hsub_split.size(), -1);
        const int nl = (int)lwho.size();
        const std::vector<int32_t> ord = by_length(llen, kHubPieceCap);
        const int first = (int)hcptr.size() - 1;
        for (int c = 0; c * 32 < nl; ++c) {
            int32_t w = 0;
            for (int l = 0; l < 32; ++l) {
                const int i = c * 32 + l;
                if (i >= nl) {
                    hcrow.push_back(-1);
                    continue;
                }
                const int li = ord[(size_t)i];
                const int who = lwho[(size_t)li];
                hcrow.push_back(who);
                if (who >= 0)
                    hbase[(size_t)sl * n + who] = helems + l;
                else
                    subbase[(size_t)(-who - 2)] = helems + l;
                w = std::max(w, llen[(size_t)li]);
            }
            helems += 32 * (int64_t)w;
            if (helems >= (int64_t(1) << 31) - 64) return LILAC_OK;  // offsets overflow: not built
            hcptr.push_back((int32_t)helems);
        }
        // G runs of about equal work: elements plus kHubChunkCost per chunk
        const int cb = first, ce = (int)hcptr.size() - 1;
        auto work = [&](int ch) { return (int64_t)hcptr[(size_t)ch] + kHubChunkCost * (int64_t)ch; };
        int cur = cb;
        for (int jr = 0; jr < G; ++jr) {
            int nxt = ce;
            if (jr < G - 1) {
                const int64_t target = work(cb) + (work(ce) - work(cb)) * (jr + 1) / G;
                nxt = cur;
                while (nxt < ce && work(nxt + 1) <= target) ++nxt;
            }
            ranges.push_back(make_int4(sl, cur, nxt, 0));
            cur = nxt;
        }
    }
    std::vector<int32_t> hperm((size_t)helems, -1);
    std::vector<uint16_t> hcol((size_t)helems, (uint16_t)W);
    // cold part: lanes are rows, or pieces of at most `cap` of a longer row
    const double cmean = n > 0 ? (double)(nnz - (int64_t)std::accumulate(plen.begin(), plen.end(), int64_t(0))) / n : 0.0;
    int cap = 32;
    while (cap < 4.0 * cmean && cap < 4096) cap *= 2;
    std::vector<int32_t> who, len;
    who.reserve((size_t)n);
    len.reserve((size_t)n);
    std::vector<int4> splits;
    std::vector<int32_t> piece_split, first_lane((size_t)n, -1), csplit_of((size_t)n, -1);
    for (int r = 0; r < n; ++r) {
        const int L = clen[(size_t)r];
        first_lane[(size_t)r] = (int)who.size();
        if (L <= cap) {
            who.push_back(r);
            len.push_back(L);
            continue;
        }
        const int lid = (int)splits.size();
        csplit_of[(size_t)r] = lid;
        const int np = (L + cap - 1) / cap;
        const int firstp = (int)piece_split.size();
        splits.push_back(make_int4(r, firstp, np, row_mask(r)));
        for (int j = 0; j < np; ++j) {
            piece_split.push_back(lid);
            who.push_back(-(2 + firstp + j));
            len.push_back(std::min(cap, L - j * cap));
        }
    }
    const int64_t V = (int64_t)who.size();
    if (V >= (int64_t(1) << 31) / 32) return LILAC_OK;
    const std::vector<int32_t> cord = by_length(len, cap);
    const int nch = (int)((V + 31) / 32);
    std::vector<int32_t> ccptr((size_t)nch + 1, 0), ccrow((size_t)nch * 32, -1);
    std::vector<uint8_t> cmask((size_t)nch * 32, 0);
    std::vector<int64_t> lane_base((size_t)V);
    std::vector<int32_t> lane_pos((size_t)V);
    for (int c = 0; c < nch; ++c) {
        int32_t w = 0;
        for (int l = 0; l < 32; ++l) {
            const int64_t i = (int64_t)c * 32 + l;
            if (i >= V) break;
            const int32_t li = cord[(size_t)i];
            lane_pos[(size_t)li] = (int32_t)i;
            ccrow[(size_t)i] = who[(size_t)li];
            if (who[(size_t)li] >= 0) cmask[(size_t)i] = (uint8_t)row_mask(who[(size_t)li]);
            lane_base[(size_t)li] = (int64_t)ccptr[(size_t)c] + l;
            w = std::max(w, len[(size_t)li]);
        }
        const int64_t e = (int64_t)ccptr[(size_t)c] + 32 * (int64_t)w;
        if (e >= (int64_t(1) << 31) - 64) return LILAC_OK;
        ccptr[(size_t)c + 1] = (int32_t)e;
    }
    const int64_t celems = ccptr[(size_t)nch];
    // the slab partials of a row go where the cold copy reads them: at its
    // lane's position, or after all lanes for a split row
    const int pstride = 32 * nch + (int)splits.size();
    auto ppos = [&](int r) {
        const int lid = csplit_of[(size_t)r];
        return lid >= 0 ? 32 * nch + lid : lane_pos[(size_t)first_lane[(size_t)r]];
    };
    for (auto& v : hcrow)
        if (v >= 0) v = ppos(v);
    for (auto& q : hsplits) q.x = ppos(q.x);
    std::vector<int32_t> cperm((size_t)celems, -1), ccol((size_t)celems, -1);
    {
        std::vector<int32_t> fill((size_t)S);
        for (int r = 0; r < n; ++r) {
            std::fill(fill.begin(), fill.end(), 0);
            int j = 0;  // cold elements of the row so far
            for (int k = rp[r]; k < rp[r + 1]; ++k) {
                const int c = col[(size_t)k];
                const int h = slot[(size_t)c];
                if (h >= 0) {
                    const int sl = h / W;
                    const int e = fill[(size_t)sl]++;
                    const int lid = hsplit_of[(size_t)sl * n + r];
                    const int64_t q =
                        lid < 0 ? hbase[(size_t)sl * n + r] + 32 * (int64_t)e
                                : subbase[(size_t)(hsplits[(size_t)lid].y + e / kHubPieceCap)] +
                                      32 * (int64_t)(e % kHubPieceCap);
                    hperm[(size_t)q] = k;
                    hcol[(size_t)q] = (uint16_t)(h - sl * W);
                } else {
                    const int lane = first_lane[(size_t)r] + j / cap * (clen[(size_t)r] > cap ? 1 : 0);
                    const int pos = clen[(size_t)r] > cap ? j % cap : j;
                    const int64_t q = lane_base[(size_t)lane] + 32 * (int64_t)pos;
                    cperm[(size_t)q] = k;
                    ccol[(size_t)q] = c;
                    ++j;
                }
            }
        }
    }
    const size_t hpad = (size_t)helems + 64, cpad = (size_t)celems + 64;
    const size_t nsplit = splits.size(), npieces = piece_split.size();
    LILAC_TRY(A->ws_alloc(A->hub_cols, sizeof(int32_t) * (size_t)H));
    LILAC_TRY(A->ws_alloc(A->hub_xhot, vsz * ((size_t)H + 8)));
    LILAC_TRY(A->ws_alloc(A->hub_cptr, sizeof(int32_t) * hcptr.size()));
    LILAC_TRY(A->ws_alloc(A->hub_crow, sizeof(int32_t) * hcrow.size()));
    LILAC_TRY(A->ws_alloc(A->hub_col, sizeof(uint16_t) * hpad));
    LILAC_TRY(A->ws_alloc(A->hub_val, vsz * hpad));
    LILAC_TRY(A->ws_alloc(A->hub_perm, sizeof(int32_t) * std::max<size_t>(1, (size_t)helems)));
    LILAC_TRY(A->ws_alloc(A->hub_ranges, sizeof(int4) * ranges.size()));
    LILAC_TRY(A->ws_alloc(A->hub_P, sizeof(double) * (size_t)S * (size_t)std::max(1, pstride)));
    const size_t nhs = hsplits.size(), nsub = hsub_split.size();
    LILAC_TRY(A->ws_alloc(A->hub_splits, sizeof(int4) * std::max<size_t>(1, nhs)));
    LILAC_TRY(A->ws_alloc(A->hub_sub_split, sizeof(int32_t) * std::max<size_t>(1, nsub)));
    LILAC_TRY(A->ws_alloc(A->hub_part, sizeof(double) * std::max<size_t>(1, nsub)));
    LILAC_TRY(A->ws_alloc(A->hub_cnt, sizeof(unsigned) * std::max<size_t>(1, nhs)));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hub_cnt.p, 0, A->hub_cnt.bytes, s));
    LILAC_TRY(A->ws_alloc(A->hubc_cptr, sizeof(int32_t) * ccptr.size()));
    LILAC_TRY(A->ws_alloc(A->hubc_crow, sizeof(int32_t) * ccrow.size()));
    LILAC_TRY(A->ws_alloc(A->hubc_col, sizeof(int32_t) * cpad));
    LILAC_TRY(A->ws_alloc(A->hubc_val, vsz * cpad));
    LILAC_TRY(A->ws_alloc(A->hubc_perm, sizeof(int32_t) * std::max<size_t>(1, (size_t)celems)));
    LILAC_TRY(A->ws_alloc(A->hubc_splits, sizeof(int4) * std::max<size_t>(1, nsplit)));
    LILAC_TRY(A->ws_alloc(A->hubc_piece_split, sizeof(int32_t) * std::max<size_t>(1, npieces)));
    LILAC_TRY(A->ws_alloc(A->hubc_part, sizeof(double) * std::max<size_t>(1, npieces)));
    LILAC_TRY(A->ws_alloc(A->hubc_red, sizeof(double) * kMaxRed * std::max<size_t>(1, nsplit)));
    LILAC_TRY(A->ws_alloc(A->hubc_cnt, sizeof(unsigned) * std::max<size_t>(1, nsplit)));
    LILAC_TRY(A->ws_alloc(A->hubc_mask, cmask.size()));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hub_val.p, 0, A->hub_val.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hub_col.p, 0, A->hub_col.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hubc_val.p, 0, A->hubc_val.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hubc_col.p, 0xff, A->hubc_col.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hubc_part.p, 0, A->hubc_part.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hubc_red.p, 0, A->hubc_red.bytes, s));
    LILAC_CUDA_TRY(cudaMemsetAsync(A->hubc_cnt.p, 0, A->hubc_cnt.bytes, s));
    auto up = [&](lilac::DevBuf& d, const void* h, size_t bytes) -> lilac_status {
        if (bytes) LILAC_CUDA_TRY(cudaMemcpyAsync(d.p, h, bytes, cudaMemcpyHostToDevice, s));
        return LILAC_OK;
    };
    LILAC_TRY(up(A->hub_cols, hot.data(), sizeof(int32_t) * hot.size()));
    LILAC_TRY(up(A->hub_cptr, hcptr.data(), sizeof(int32_t) * hcptr.size()));
    LILAC_TRY(up(A->hub_crow, hcrow.data(), sizeof(int32_t) * hcrow.size()));
    LILAC_TRY(up(A->hub_col, hcol.data(), sizeof(uint16_t) * hcol.size()));
    LILAC_TRY(up(A->hub_perm, hperm.data(), sizeof(int32_t) * hperm.size()));
    LILAC_TRY(up(A->hub_ranges, ranges.data(), sizeof(int4) * ranges.size()));
    LILAC_TRY(up(A->hub_splits, hsplits.data(), sizeof(int4) * nhs));
    LILAC_TRY(up(A->hub_sub_split, hsub_split.data(), sizeof(int32_t) * nsub));
    LILAC_TRY(up(A->hubc_cptr, ccptr.data(), sizeof(int32_t) * ccptr.size()));
    LILAC_TRY(up(A->hubc_crow, ccrow.data(), sizeof(int32_t) * ccrow.size()));
    LILAC_TRY(up(A->hubc_col, ccol.data(), sizeof(int32_t) * ccol.size()));
    LILAC_TRY(up(A->hubc_perm, cperm.data(), sizeof(int32_t) * cperm.size()));
    LILAC_TRY(up(A->hubc_splits, splits.data(), sizeof(int4) * nsplit));
    LILAC_TRY(up(A->hubc_piece_split, piece_split.data(), sizeof(int32_t) * npieces));
    LILAC_TRY(up(A->hubc_mask, cmask.data(), cmask.size()));
    A->hub_H = H;
    A->hub_S = S;
    A->hub_W = W;
    A->hub_grid = (int)ranges.size();
    A->hub_pstride = pstride;
    A->hub_elems = helems;
    A->hubc_elems = celems;
    A->hubc_nchunks = nch;
    A->hubc_nsplit = (int)nsplit;
    A->hubc_npieces = (int)npieces;
    A->hub_share = share[S];
    A->hub_two_pass = n >= (1 << 16) && cmean < 64.0;
    LILAC_TRY(A->dtype == LILAC_F64 ? hub_regather<double>(A, s) : hub_regather<float>(A, s));
    // the host vectors above must outlive the copies
    LILAC_CUDA_TRY(cudaStreamSynchronize(s));
    A->hub_built = true;
    return LILAC_OK;
}

lilac_status hub_refresh_values(lilac_csr A, cudaStream_t s) {
    if (!A->hub_built) return LILAC_OK;
    return A->dtype == LILAC_F64 ? hub_regather<double>(A, s) : hub_regather<float>(A, s);
}

lilac_status hub_zero_counters(lilac_csr A, cudaStream_t s) {
    if (A->hubc_cnt.p) LILAC_CUDA_TRY(cudaMemsetAsync(A->hubc_cnt.p, 0, A->hubc_cnt.bytes, s));
    if (A->hub_cnt.p) LILAC_CUDA_TRY(cudaMemsetAsync(A->hub_cnt.p, 0, A->hub_cnt.bytes, s));
    return LILAC_OK;
}

void hub_release(lilac_csr A) {
    lilac::DevBuf* b[] = {&A->hub_cols,   &A->hub_xhot,    &A->hub_cptr,        &A->hub_crow,
                          &A->hub_col,    &A->hub_val,     &A->hub_perm,        &A->hub_ranges,
                          &A->hub_P,      &A->hubc_cptr,   &A->hubc_crow,       &A->hubc_col,
                          &A->hubc_val,   &A->hubc_perm,   &A->hubc_splits,     &A->hubc_piece_split,
                          &A->hubc_part,  &A->hubc_red,    &A->hubc_cnt,        &A->hubc_mask,
                          &A->hub_splits, &A->hub_sub_split, &A->hub_part,      &A->hub_cnt};
    for (auto* d : b) d->release();
    A->hub_H = A->hub_S = A->hub_W = A->hub_grid = A->hub_pstride = 0;
    A->hub_elems = A->hubc_elems = 0;
    A->hubc_nchunks = A->hubc_nsplit = A->hubc_npieces = 0;
    A->hub_share = 0.0;
    A->hub_two_pass = false;
    A->hub_built = false;
}

lilac_status ensure_hub(lilac_csr A, cudaStream_t s) {
    if (A->hub_built || !hub_worthwhile(A)) return LILAC_OK;
    return build_hub(A, s);
}

}  // namespace lilac
