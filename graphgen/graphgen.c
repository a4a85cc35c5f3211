/*
 * Seeded synthetic graph generators shared by the tests, the CUDA path's
 * callers and the oracle.  This file draws inputs only: it holds none of the
 * shortest-path or pruning arithmetic.
 *
 * Every random number is a pure function of (seed, stream, counter) through
 * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014; finaliser constants as published by Vigna), so
 * the parallel loops below give the same bytes on any core count and on both
 * x86_64 and aarch64.
 *
 * Workload shapes follow the experiment section of the paper (synthetic
 * graphs, integer weights drawn uniformly) and the five workload recipes of
 * this library: Erdos-Renyi G(n,M), R-MAT, a 4-neighbour grid, a batched
 * mix and fp32 jittered weights.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GG_STREAM_PERM 1u
#define GG_STREAM_W 2u
#define GG_STREAM_RMAT 3u
#define GG_STREAM_ER 4u
#define GG_STREAM_GRID_H 5u
#define GG_STREAM_GRID_V 6u
#define GG_STREAM_SRC 7u
#define GG_STREAM_NORMAL 8u
#define GG_STREAM_JITTER 9u
#define GG_STREAM_BATCH 10u

static inline uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* counter-based draw: a pure function of its three arguments */
static inline uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return sm64(sm64(seed ^ (stream * 0xD1B54A32D192ED03ULL)) ^ ctr);
}

uint64_t gg_rand_u64(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return gg_rand(seed, stream, ctr);
}

/* uniform integer in [lo, hi] (inclusive), multiply-shift on the top 32 bits */
static inline uint32_t gg_uint(uint64_t r, uint32_t lo, uint32_t hi) {
    uint64_t range = (uint64_t)hi - lo + 1u;
    return lo + (uint32_t)(((r >> 32) * range) >> 32);
}

/* uniform double in [0, 1) from the top 53 bits */
static inline double gg_unit(uint64_t r) {
    return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------- weights */

/* w[i] = U{lo..hi}, drawn from edge counter i */
void gg_weights_u32(uint64_t seed, uint64_t n, uint32_t lo, uint32_t hi, uint32_t* w) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) w[i] = gg_uint(gg_rand(seed, GG_STREAM_W, (uint64_t)i), lo, hi);
}

/* w[i] = fp32( lo + (hi-lo)*U + jitter*U' ), U, U' in [0,1) */
void gg_weights_f32(uint64_t seed, uint64_t n, double lo, double hi, double jitter, float* w) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) {
        double a = gg_unit(gg_rand(seed, GG_STREAM_W, (uint64_t)i));
        double b = gg_unit(gg_rand(seed, GG_STREAM_JITTER, (uint64_t)i));
        w[i] = (float)(lo + (hi - lo) * a + jitter * b);
    }
}

/* standard normal via Box-Muller on two counter draws */
void gg_normal_f32(uint64_t seed, uint64_t n, float* out) {
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)n; ++i) {
        double u1 = gg_unit(gg_rand(seed, GG_STREAM_NORMAL, 2u * (uint64_t)i));
        double u2 = gg_unit(gg_rand(seed, GG_STREAM_NORMAL, 2u * (uint64_t)i + 1u));
        if (u1 < 1e-300) u1 = 1e-300;
        out[i] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
}

/* ------------------------------------------------------------ permutation */

/* Fisher-Yates shuffle of 0..n-1 */
void gg_permutation(uint64_t seed, uint32_t n, uint32_t* perm) {
    uint32_t i;
    for (i = 0; i < n; ++i) perm[i] = i;
    if (n < 2) return;
    for (i = n - 1; i > 0; --i) {
        uint32_t j = (uint32_t)(((gg_rand(seed, GG_STREAM_PERM, i) >> 32) * (uint64_t)(i + 1u)) >> 32);
        uint32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

/* ------------------------------------------------------------------ R-MAT */

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): every edge descends `scale`
 * levels of the adjacency matrix, picking quadrant (0,0),(0,1),(1,0),(1,1)
 * with probabilities a, b, c, 1-a-b-c.  Endpoints >= n are redrawn (n <
 * 2^scale for the batched mix).  If `permute`, vertex ids are relabelled by
 * a seeded permutation so that id blocks are not degree-sorted.  Duplicates
 * and self-loops are kept: the edge list is raw.
 */
void gg_rmat(uint64_t seed, uint32_t scale, uint32_t n, uint64_t nedges, double a, double b, double c,
             int permute, uint32_t* src, uint32_t* dst) {
    uint32_t* perm = NULL;
    int64_t i;
    if (permute) {
        perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
        gg_permutation(seed, n, perm);
    }
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)nedges; ++i) {
        uint64_t attempt = 0;
        for (;;) {
            uint32_t s = 0, d = 0, lvl;
            for (lvl = 0; lvl < scale; ++lvl) {
                double p = gg_unit(gg_rand(seed ^ (attempt * 0x9E3779B97F4A7C15ULL), GG_STREAM_RMAT,
                                           (uint64_t)i * 64u + lvl));
                uint32_t bit = scale - 1u - lvl;
                if (p < a) {
                } else if (p < a + b) {
                    d |= 1u << bit;
                } else if (p < a + b + c) {
                    s |= 1u << bit;
                } else {
                    s |= 1u << bit;
                    d |= 1u << bit;
                }
            }
            if (s < n && d < n) {
                src[i] = perm ? perm[s] : s;
                dst[i] = perm ? perm[d] : d;
                break;
            }
            ++attempt;
        }
    }
    free(perm);
}

/* --------------------------------------------------------- Erdos-Renyi G(n,M) */

/*
 * M distinct (src,dst) pairs with src != dst, by rejection: candidate k is
 * drawn from counter k; loops and repeats are rejected with an open-address
 * hash set.  Accepted pairs are emitted in acceptance order.
 * Returns 0, or -1 if M exceeds n(n-1).
 */
int gg_er(uint64_t seed, uint32_t n, uint64_t M, uint32_t* src, uint32_t* dst) {
    uint64_t cap = 1, mask, k = 0, got = 0;
    uint64_t* table;
    if (n < 2 || M > (uint64_t)n * (uint64_t)(n - 1u)) return -1;
    while (cap < 2 * M + 16) cap <<= 1;
    mask = cap - 1;
    table = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cap);
    memset(table, 0xFF, sizeof(uint64_t) * (size_t)cap);
    while (got < M) {
        uint64_t r = gg_rand(seed, GG_STREAM_ER, k++);
        uint32_t s = (uint32_t)(((r >> 32) * (uint64_t)n) >> 32);
        uint32_t d = (uint32_t)(((r & 0xFFFFFFFFu) * (uint64_t)n) >> 32);
        uint64_t key, h;
        if (s == d) continue;
        key = ((uint64_t)s << 32) | d;
        h = sm64(key) & mask;
        while (table[h] != UINT64_MAX && table[h] != key) h = (h + 1) & mask;
        if (table[h] == key) continue;
        table[h] = key;
        src[got] = s;
        dst[got] = d;
        ++got;
    }
    free(table);
    return 0;
}

/* ------------------------------------------------------------------- grid */

/*
 * rows x cols 4-neighbour grid, v = r*cols + c, both directions of every
 * undirected edge.  One weight per undirected edge (symmetric), U{lo..hi}.
 * Emits 2*(rows*(cols-1) + (rows-1)*cols) edges in vertex order.
 */
uint64_t gg_grid(uint64_t seed, uint32_t rows, uint32_t cols, uint32_t lo, uint32_t hi,
                 uint32_t* src, uint32_t* dst, uint32_t* w) {
    int64_t r;
    /* per-vertex emission offsets are closed-form, so rows can run in parallel */
#pragma omp parallel for schedule(static)
    for (r = 0; r < (int64_t)rows; ++r) {
        uint32_t c;
        /* edges emitted before row r: every earlier row emits its full count */
        uint64_t per_row_full = 2ull * (cols - 1u) + 2ull * cols; /* horizontal both dirs + vertical both dirs */
        uint64_t pos = (uint64_t)r * per_row_full;
        /* vertical edges of a row are counted toward the upper row, so the last row emits fewer */
        for (c = 0; c < cols; ++c) {
            uint32_t v = (uint32_t)r * cols + c;
            if (c + 1u < cols) {
                uint32_t wt = gg_uint(gg_rand(seed, GG_STREAM_GRID_H, v), lo, hi);
                src[pos] = v; dst[pos] = v + 1u; w[pos] = wt; ++pos;
                src[pos] = v + 1u; dst[pos] = v; w[pos] = wt; ++pos;
            }
            if ((uint32_t)r + 1u < rows) {
                uint32_t wt = gg_uint(gg_rand(seed, GG_STREAM_GRID_V, v), lo, hi);
                src[pos] = v; dst[pos] = v + cols; w[pos] = wt; ++pos;
                src[pos] = v + cols; dst[pos] = v; w[pos] = wt; ++pos;
            }
        }
    }
    return 2ull * ((uint64_t)rows * (cols - 1u) + (uint64_t)(rows - 1u) * cols);
}

/* ---------------------------------------------------------------- sources */

/*
 * `count` distinct vertices with at least one out-edge that is not a
 * self-loop, drawn uniformly with counter k = 0,1,...  Returns the number
 * found (fewer only if the graph has fewer such vertices).
 */
uint32_t gg_pick_sources(uint64_t seed, uint32_t n, uint64_t E, const uint32_t* src, const uint32_t* dst,
                         uint32_t count, uint32_t* out) {
    uint8_t* ok = (uint8_t*)calloc(n ? n : 1, 1);
    uint64_t e, k = 0, eligible = 0;
    uint32_t got = 0;
    for (e = 0; e < E; ++e)
        if (src[e] != dst[e] && src[e] < n && !ok[src[e]]) { ok[src[e]] = 1; ++eligible; }
    if (count > eligible) count = (uint32_t)eligible;
    while (got < count) {
        uint32_t v = (uint32_t)(((gg_rand(seed, GG_STREAM_SRC, k++) >> 32) * (uint64_t)n) >> 32);
        if (ok[v] == 1) { ok[v] = 2; out[got++] = v; }
    }
    free(ok);
    return got;
}

/* ------------------------------------------------------------ batched mix */

/*
 * Parameters of graph g of a batched mix: type (0 = Erdos-Renyi out-degree 8,
 * 1 = R-MAT edge factor 8) by a fair coin, vertex count round(2^U(lo_exp,hi_exp)).
 */
void gg_batch_params(uint64_t seed, uint32_t g, double lo_exp, double hi_exp, uint32_t* type, uint32_t* n) {
    uint64_t r0 = gg_rand(seed, GG_STREAM_BATCH, 2u * (uint64_t)g);
    uint64_t r1 = gg_rand(seed, GG_STREAM_BATCH, 2u * (uint64_t)g + 1u);
    double x = lo_exp + (hi_exp - lo_exp) * gg_unit(r1);
    *type = (uint32_t)(r0 >> 63);
    *n = (uint32_t)floor(pow(2.0, x) + 0.5);
}

/* seed of member g of a batch */
uint64_t gg_member_seed(uint64_t seed, uint32_t g) { return sm64(seed ^ sm64(0xBA7C400000000000ULL + g)); }
