/*
 * Seeded synthetic inputs shared by the CUDA library's tests/benchmarks and
 * by the CPU oracle's tests.  This file holds input construction only (matrix
 * structure, matrix values and vectors); none of the sparse linear algebra
 * that the library or the oracle computes lives here.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), used as a counter-based
 * generator: draw k of a stream with key s is mix(s + (k+1)*0x9E3779B97F4A7C15).
 * A uniform double in [0,1) is (z >> 11) * 2^-53.
 *
 * Every generator writes int32 CSR (row_ptr[n+1], col_ind[nnz]) with the
 * columns of a row in ascending order, and returns nnz (or -1 on a size
 * overflow).  Callers allocate the output arrays at the documented bound.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw k of stream `key`. */
static inline uint64_t sm64_at(uint64_t key, uint64_t k) {
    return sm64_mix(key + (k + 1) * SM64_GAMMA);
}

static inline double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

/* Key of sub-stream `id` of a user seed (so that, e.g., the R-MAT edge draws
 * and the vertex relabelling never share draws). */
static inline uint64_t stream_key(uint64_t seed, uint64_t id) {
    return sm64_mix(seed ^ (id * 0xD1B54A32D192ED03ULL));
}

uint64_t gen_splitmix64_at(uint64_t key, uint64_t k) { return sm64_at(key, k); }

/* out[i] = lo + (hi - lo) * u_i, u_i = draw i of stream `seed` (the seed is
 * the stream key itself, so seed 0 gives the documented x of the 2D
 * Laplacian workload).  For [-1, 1] this is 2u - 1 exactly. */
void gen_uniform_f64(uint64_t seed, int64_t n, double lo, double hi, double* out) {
    double w = hi - lo;
    for (int64_t i = 0; i < n; ++i) out[i] = lo + w * u01(sm64_at(seed, (uint64_t)i));
}

void gen_uniform_f32(uint64_t seed, int64_t n, double lo, double hi, float* out) {
    double w = hi - lo;
    for (int64_t i = 0; i < n; ++i) out[i] = (float)(lo + w * u01(sm64_at(seed, (uint64_t)i)));
}

/* 2D 5-point Laplacian on an m x m grid with Dirichlet boundary, natural
 * (row-major) ordering i = a*m + b.  Diagonal 4, -1 to N/S/E/W neighbours.
 * nnz = 5m^2 - 4m.  vals_f64 and/or vals_f32 may be NULL. */
int64_t gen_laplacian2d(int32_t m, int32_t* row_ptr, int32_t* col_ind,
                        double* vals_f64, float* vals_f32) {
    int64_t k = 0;
    row_ptr[0] = 0;
    for (int32_t a = 0; a < m; ++a)
        for (int32_t b = 0; b < m; ++b) {
            int32_t i = a * m + b;
            int32_t cols[5];
            double v[5];
            int c = 0;
            if (a > 0)     { cols[c] = i - m; v[c++] = -1.0; }
            if (b > 0)     { cols[c] = i - 1; v[c++] = -1.0; }
            cols[c] = i; v[c++] = 4.0;
            if (b < m - 1) { cols[c] = i + 1; v[c++] = -1.0; }
            if (a < m - 1) { cols[c] = i + m; v[c++] = -1.0; }
            for (int t = 0; t < c; ++t, ++k) {
                col_ind[k] = cols[t];
                if (vals_f64) vals_f64[k] = v[t];
                if (vals_f32) vals_f32[k] = (float)v[t];
            }
            row_ptr[i + 1] = (int32_t)k;
        }
    return k;
}

/* 3D 7-point Laplacian on an m^3 grid, i = (a*m + b)*m + c, diagonal 6.
 * nnz = 7m^3 - 6m^2. */
int64_t gen_laplacian3d(int32_t m, int32_t* row_ptr, int32_t* col_ind,
                        double* vals_f64, float* vals_f32) {
    int64_t k = 0;
    int64_t mm = (int64_t)m * m;
    row_ptr[0] = 0;
    for (int32_t a = 0; a < m; ++a)
        for (int32_t b = 0; b < m; ++b)
            for (int32_t c = 0; c < m; ++c) {
                int64_t i = ((int64_t)a * m + b) * m + c;
                int64_t cols[7];
                double v[7];
                int t = 0;
                if (a > 0)     { cols[t] = i - mm; v[t++] = -1.0; }
                if (b > 0)     { cols[t] = i - m;  v[t++] = -1.0; }
                if (c > 0)     { cols[t] = i - 1;  v[t++] = -1.0; }
                cols[t] = i; v[t++] = 6.0;
                if (c < m - 1) { cols[t] = i + 1;  v[t++] = -1.0; }
                if (b < m - 1) { cols[t] = i + m;  v[t++] = -1.0; }
                if (a < m - 1) { cols[t] = i + mm; v[t++] = -1.0; }
                for (int q = 0; q < t; ++q, ++k) {
                    col_ind[k] = (int32_t)cols[q];
                    if (vals_f64) vals_f64[k] = v[q];
                    if (vals_f32) vals_f32[k] = (float)v[q];
                }
                row_ptr[i + 1] = (int32_t)k;
            }
    return k;
}

/* --- helpers: sort (row, col) COO entries ------------------------------ */

typedef struct { int32_t r, c; double v; } coo_t;

static int coo_cmp(const void* pa, const void* pb) {
    const coo_t* a = (const coo_t*)pa;
    const coo_t* b = (const coo_t*)pb;
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return 0;
}

/*
 * Random symmetric positive definite matrix shaped like the NAS CG matrix
 * (uniformly random columns).  Row i draws k distinct columns j != i, each
 * with a value U[0,1) (column draw: floor(u*n), redrawn on a clash; then one
 * value draw), all from one stream in row order.  A = B + B^T (a pair present
 * in both B_ij and B_ji is summed), then a_ii = sum_{j != i} a_ij + shift,
 * the off-diagonal sum taken in ascending column order.  Strict diagonal
 * dominance with a positive diagonal makes A SPD.
 * Output bound: nnz <= n*(2k+1).  If vals_f32 is set, values are also
 * written rounded to FP32.
 */
int64_t gen_spd_random(int32_t n, int32_t k, double shift, uint64_t seed,
                       int32_t* row_ptr, int32_t* col_ind, double* vals_f64, float* vals_f32) {
    if (k >= n) return -1;
    int64_t nb = (int64_t)n * k;
    coo_t* e = (coo_t*)malloc(sizeof(coo_t) * (size_t)(2 * nb));
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!e || !mark) { free(e); free(mark); return -1; }
    for (int32_t i = 0; i < n; ++i) mark[i] = -1;
    uint64_t draw = 0;
    int64_t t = 0;
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t q = 0; q < k; ++q) {
            int32_t j;
            for (;;) {
                j = (int32_t)(u01(sm64_at(seed, draw++)) * (double)n);
                if (j >= n) j = n - 1;
                if (j != i && mark[j] != i) break;
            }
            mark[j] = i;
            double v = u01(sm64_at(seed, draw++));
            e[t].r = i; e[t].c = j; e[t].v = v; ++t;
            e[t].r = j; e[t].c = i; e[t].v = v; ++t;
        }
    }
    qsort(e, (size_t)t, sizeof(coo_t), coo_cmp);
    /* merge duplicates; insert diagonal */
    int64_t nz = 0;
    int64_t p = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t row_start = nz;
        int64_t diag_pos = -1;
        double offsum = 0.0;
        int diag_done = 0;
        while (p < t && e[p].r == i) {
            int32_t c = e[p].c;
            double v = e[p].v;
            ++p;
            while (p < t && e[p].r == i && e[p].c == c) { v += e[p].v; ++p; }
            if (!diag_done && c > i) {
                diag_pos = nz; col_ind[nz] = i; vals_f64[nz] = 0.0; ++nz; diag_done = 1;
            }
            col_ind[nz] = c; vals_f64[nz] = v; ++nz;
        }
        if (!diag_done) { diag_pos = nz; col_ind[nz] = i; vals_f64[nz] = 0.0; ++nz; }
        for (int64_t q = row_start; q < nz; ++q)
            if (q != diag_pos) offsum += vals_f64[q];
        vals_f64[diag_pos] = offsum + shift;
        row_ptr[i + 1] = (int32_t)nz;
    }
    if (vals_f32)
        for (int64_t q = 0; q < nz; ++q) vals_f32[q] = (float)vals_f64[q];
    free(e);
    free(mark);
    return nz;
}

/*
 * Symmetric banded SPD matrix: full band |i-j| <= w.  For each i and each
 * j in (i, i+w] one value U[0,1) is drawn (row-major order of the upper
 * triangle), optionally rounded to FP32 first (fp32_exact != 0), and placed
 * at (i,j) and (j,i).  a_ii = (sum of the off-diagonals of row i in
 * ascending column order) + shift.  Output bound: nnz <= n*(2w+1).
 */
int64_t gen_banded_spd(int32_t n, int32_t w, double shift, uint64_t seed, int fp32_exact,
                       int32_t* row_ptr, int32_t* col_ind, double* vals_f64, float* vals_f32) {
    if (w < 0) return -1;
    /* upper[i*w + (j-i-1)] holds the value of (i, j) */
    double* upper = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(w > 0 ? w : 1));
    if (!upper) return -1;
    uint64_t draw = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t d = 1; d <= w; ++d) {
            double v = 0.0;
            if (i + d < n) {
                v = u01(sm64_at(seed, draw++));
                if (fp32_exact) v = (double)(float)v;
            }
            upper[(int64_t)i * w + (d - 1)] = v;
        }
    int64_t nz = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t lo = i - w < 0 ? 0 : i - w;
        int32_t hi = i + w >= n ? n - 1 : i + w;
        int64_t diag_pos = -1;
        double offsum = 0.0;
        for (int32_t j = lo; j <= hi; ++j) {
            double v;
            if (j < i) v = upper[(int64_t)j * w + (i - j - 1)];
            else if (j > i) v = upper[(int64_t)i * w + (j - i - 1)];
            else { diag_pos = nz; v = 0.0; }
            col_ind[nz] = j;
            vals_f64[nz] = v;
            ++nz;
        }
        for (int64_t q = row_ptr[i]; q < nz; ++q)
            if (q != diag_pos) offsum += vals_f64[q];
        vals_f64[diag_pos] = offsum + shift;
        row_ptr[i + 1] = (int32_t)nz;
    }
    if (vals_f32)
        for (int64_t q = 0; q < nz; ++q) vals_f32[q] = (float)vals_f64[q];
    free(upper);
    return nz;
}

/* --- R-MAT --------------------------------------------------------------- */

static void radix_sort_u64(uint64_t* a, uint64_t* tmp, int64_t n, int key_bits) {
    const int RB = 11;
    const int64_t NB = 1 << RB;
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)NB);
    uint64_t* src = a;
    uint64_t* dst = tmp;
    int passes = (key_bits + RB - 1) / RB;
    for (int ps = 0; ps < passes; ++ps) {
        int sh = ps * RB;
        memset(cnt, 0, sizeof(int64_t) * (size_t)NB);
        for (int64_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & (NB - 1)]++;
        int64_t s = 0;
        for (int64_t b = 0; b < NB; ++b) { int64_t c = cnt[b]; cnt[b] = s; s += c; }
        for (int64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & (NB - 1)]++] = src[i];
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(uint64_t) * (size_t)n);
    free(cnt);
}

/*
 * R-MAT graph (Chakrabarti, Zhan & Faloutsos, SDM 2004) with 2^scale vertices
 * and edge_factor*2^scale drawn edges, quadrant probabilities a, b, c and
 * d = 1-a-b-c, no per-level noise.  Edge e takes draw e*scale + l of stream
 * key(seed, 1) for level l (most significant bit first): u < a -> (0,0),
 * u < a+b -> (0,1), u < a+b+c -> (1,0), else (1,1) for (src bit, dst bit).
 * If permute != 0, both endpoints are relabelled by one Fisher-Yates
 * permutation of the vertices, drawn from stream key(seed, 2) (step t swaps
 * slot N-1-t with slot floor(u_t * (N-t))).  Self-loops and duplicate edges
 * are removed.  Output: the TRANSPOSED adjacency in CSR (row = destination,
 * column = source, columns ascending), values 1/outdeg(source) rounded to
 * FP32 (outdeg counts unique non-loop out-edges), and outdeg[N].
 * Output bound: nnz <= edge_factor * 2^scale.
 */
int64_t gen_rmat_transposed(int32_t scale, int32_t edge_factor, double a, double b, double c,
                            uint64_t seed, int permute,
                            int32_t* row_ptr, int32_t* col_ind, float* vals, int32_t* outdeg) {
    if (scale < 1 || scale > 30) return -1;
    int64_t N = (int64_t)1 << scale;
    int64_t M = (int64_t)edge_factor * N;
    if (M >= ((int64_t)1 << 31)) return -1;
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)M);
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)M);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    if (!key || !tmp || !perm) { free(key); free(tmp); free(perm); return -1; }
    uint64_t ek = stream_key(seed, 1);
    uint64_t pk = stream_key(seed, 2);
    double ab = a + b, abc = a + b + c;
    for (int64_t i = 0; i < N; ++i) perm[i] = (int32_t)i;
    if (permute) {
        for (int64_t t = 0; t < N - 1; ++t) {
            int64_t i = N - 1 - t;
            int64_t j = (int64_t)(u01(sm64_at(pk, (uint64_t)t)) * (double)(i + 1));
            if (j > i) j = i;
            int32_t x = perm[i]; perm[i] = perm[j]; perm[j] = x;
        }
    }
    int64_t m = 0;
    for (int64_t e = 0; e < M; ++e) {
        uint64_t src = 0, dst = 0;
        uint64_t base = (uint64_t)e * (uint64_t)scale;
        for (int32_t l = 0; l < scale; ++l) {
            double u = u01(sm64_at(ek, base + (uint64_t)l));
            uint64_t sb, db;
            if (u < a) { sb = 0; db = 0; }
            else if (u < ab) { sb = 0; db = 1; }
            else if (u < abc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            src = (src << 1) | sb;
            dst = (dst << 1) | db;
        }
        if (src == dst) continue;
        uint64_t ps = (uint64_t)perm[src], pd = (uint64_t)perm[dst];
        key[m++] = (pd << scale) | ps; /* sort by (destination, source) */
    }
    radix_sort_u64(key, tmp, m, 2 * scale);
    /* unique */
    int64_t u = 0;
    for (int64_t i = 0; i < m; ++i)
        if (i == 0 || key[i] != key[i - 1]) key[u++] = key[i];
    uint64_t mask = ((uint64_t)1 << scale) - 1;
    memset(outdeg, 0, sizeof(int32_t) * (size_t)N);
    for (int64_t i = 0; i < u; ++i) outdeg[key[i] & mask]++;
    memset(row_ptr, 0, sizeof(int32_t) * (size_t)(N + 1));
    for (int64_t i = 0; i < u; ++i) row_ptr[(key[i] >> scale) + 1]++;
    for (int64_t r = 0; r < N; ++r) row_ptr[r + 1] += row_ptr[r];
    for (int64_t i = 0; i < u; ++i) {
        int32_t s = (int32_t)(key[i] & mask);
        col_ind[i] = s;
        vals[i] = (float)(1.0 / (double)outdeg[s]);
    }
    free(key); free(tmp); free(perm);
    return u;
}

/*
 * Small random CSR for edge-case tests: n rows, ncols columns, row lengths
 * drawn from [0, max_len], a fraction of rows forced empty, columns drawn
 * uniformly WITHOUT sorting and WITH possible duplicates (both allowed by
 * the CSR definition), values U[-1,1).  Output bound: nnz <= n*max_len.
 */
int64_t gen_random_csr(int32_t n, int32_t ncols, int32_t max_len, double empty_frac,
                       uint64_t seed, int32_t* row_ptr, int32_t* col_ind, double* vals) {
    uint64_t draw = 0;
    int64_t nz = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        double ue = u01(sm64_at(seed, draw++));
        int32_t len = (int32_t)(u01(sm64_at(seed, draw++)) * (double)(max_len + 1));
        if (len > max_len) len = max_len;
        if (ue < empty_frac) len = 0;
        for (int32_t q = 0; q < len; ++q) {
            int32_t c = (int32_t)(u01(sm64_at(seed, draw++)) * (double)ncols);
            if (c >= ncols) c = ncols - 1;
            col_ind[nz] = c;
            vals[nz] = 2.0 * u01(sm64_at(seed, draw++)) - 1.0;
            ++nz;
        }
        row_ptr[i + 1] = (int32_t)nz;
    }
    return nz;
}

/*
 * Power-law row lengths for load-balance tests: row i has
 * floor(max_len * u^power) entries (u uniform), so a few rows are long and
 * most are short; columns uniform (unsorted), values U[-1,1).
 */
int64_t gen_powerlaw_csr(int32_t n, int32_t ncols, int32_t max_len, int32_t power,
                         uint64_t seed, int32_t* row_ptr, int32_t* col_ind, double* vals) {
    uint64_t draw = 0;
    int64_t nz = 0;
    row_ptr[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        double u = u01(sm64_at(seed, draw++));
        double f = 1.0;
        for (int32_t q = 0; q < power; ++q) f *= u;
        int32_t len = (int32_t)((double)max_len * f);
        for (int32_t q = 0; q < len; ++q) {
            int32_t c = (int32_t)(u01(sm64_at(seed, draw++)) * (double)ncols);
            if (c >= ncols) c = ncols - 1;
            col_ind[nz] = c;
            vals[nz] = 2.0 * u01(sm64_at(seed, draw++)) - 1.0;
            ++nz;
        }
        row_ptr[i + 1] = (int32_t)nz;
    }
    return nz;
}
