/*
 * CPU oracle for the SP_Async hot path (arXiv 2103.12012).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use this file.  It shares no code with the CUDA library:
 * every function here is a plain, slow, directly checkable statement of what
 * the GPU path must produce.  Nothing is blocked, fused or reordered.
 *
 * What each function follows:
 *   orc_csr        -- the per-process adjacency Padj of Sec. III.A, made
 *                     canonical: rows sorted by head, self-loops dropped,
 *                     parallel edges collapsed to their minimum weight
 *                     (lowest original index on ties).  Distances are
 *                     unchanged by this.
 *   orc_partition  -- 1D block partitioning of Sec. III.A (read as block size
 *                     B = ceil(N/P), Pid(v) = floor(v/B)).
 *   orc_dijkstra   -- the problem statement of Sec. I (shortest s->v path
 *                     cost) computed by a textbook binary-heap Dijkstra with
 *                     lazy deletion, i.e. the priority-queue semantics of the
 *                     DIJKSTRA procedure of Sec. III.C run on the whole graph.
 *                     Partitions and messages (Sec. III.C/D) do not change the
 *                     result, so none appear here.
 *   orc_trishla    -- Algorithm 1 (Trishla, Sec. III.B), naive over all
 *                     ordered neighbour pairs, evaluated on the unpruned graph.
 *   orc_tree_grad  -- d dist(v) / d w(e) = 1 exactly when e lies on the
 *                     shortest-path tree path to v; the upstream gradient is
 *                     accumulated up the predecessor tree in decreasing
 *                     distance order.  (The paper has no gradients; this is
 *                     the derivative of the min-plus result it defines.)
 *
 * Weight types: 0 = uint32 (sums formed in 64 bits), 1 = float32 (every
 * candidate d(u)+w rounded once to float32, as the GPU path does).
 * Value conventions: unreachable dist = 0xFFFFFFFF (u32) or +inf (f32); pred
 * of the source and of unreachable vertices = 0xFFFFFFFF.  A u32 distance that
 * does not fit below 0xFFFFFFFF is reported as unreachable and the status is
 * ORC_OVERFLOW.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off (no -ffast-math).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_OVERFLOW 5

#define NONE 0xFFFFFFFFu
#define INF32 0xFFFFFFFFu

typedef struct {
    uint32_t s, d;
    uint32_t wbits;
    uint32_t id;
    int wtype;
} rec_t;

static float f32_of(uint32_t bits) {
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

static uint32_t bits_of(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

static int weight_less(uint32_t a, uint32_t b, int wtype) {
    if (wtype == 1) return f32_of(a) < f32_of(b);
    return a < b;
}

static int rec_cmp(const void* pa, const void* pb) {
    const rec_t* a = (const rec_t*)pa;
    const rec_t* b = (const rec_t*)pb;
    if (a->s != b->s) return a->s < b->s ? -1 : 1;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    if (a->wbits != b->wbits) return weight_less(a->wbits, b->wbits, a->wtype) ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

/*
 * COO -> CSR.  Out: row_ptr[V+1], col[E], w[E] (weight bits), eid[E] (index
 * of the kept edge in the input).  Returns E, or -1 on an endpoint >= V.
 */
int64_t orc_csr(uint32_t V, uint64_t E_raw, const uint32_t* src, const uint32_t* dst, const uint32_t* wbits,
                int wtype, uint32_t* row_ptr, uint32_t* col, uint32_t* w, uint32_t* eid) {
    rec_t* r;
    uint64_t i, n = 0, E = 0;
    uint32_t v;
    for (i = 0; i < E_raw; ++i)
        if (src[i] >= V || dst[i] >= V) return -1;
    r = (rec_t*)malloc(sizeof(rec_t) * (E_raw ? E_raw : 1));
    for (i = 0; i < E_raw; ++i) {
        if (src[i] == dst[i]) continue; /* self-loops never lie on a shortest path */
        r[n].s = src[i];
        r[n].d = dst[i];
        r[n].wbits = wbits[i];
        r[n].id = (uint32_t)i;
        r[n].wtype = wtype;
        ++n;
    }
    qsort(r, n, sizeof(rec_t), rec_cmp);
    for (v = 0; v <= V; ++v) row_ptr[v] = 0;
    for (i = 0; i < n; ++i) {
        if (i > 0 && r[i].s == r[i - 1].s && r[i].d == r[i - 1].d) continue; /* keep the first = minimum */
        col[E] = r[i].d;
        w[E] = r[i].wbits;
        eid[E] = r[i].id;
        row_ptr[r[i].s + 1] += 1;
        ++E;
    }
    for (v = 0; v < V; ++v) row_ptr[v + 1] += row_ptr[v];
    free(r);
    return (int64_t)E;
}

/*
 * Block partition: bounds[p] = min(p*B, V), p = 0..P, with B = ceil(V/P);
 * inter[p] = number of edges whose tail is in partition p and whose head is
 * not (the "inter-edges" of Sec. III.D).
 */
int orc_partition(uint32_t V, uint32_t P, const uint32_t* row_ptr, const uint32_t* col, uint32_t* bounds,
                  uint64_t* inter) {
    uint64_t B;
    uint32_t p, u;
    if (P == 0 || V == 0) return ORC_EINVAL;
    B = ((uint64_t)V + P - 1) / P;
    for (p = 0; p <= P; ++p) bounds[p] = (uint32_t)((uint64_t)p * B < V ? (uint64_t)p * B : V);
    for (p = 0; p < P; ++p) inter[p] = 0;
    if (row_ptr == NULL) return ORC_OK;
    for (u = 0; u < V; ++u) {
        uint32_t e;
        for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if ((uint64_t)col[e] / B != (uint64_t)u / B) inter[(uint64_t)u / B] += 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ binary heap */

typedef struct {
    double key;    /* f32 distances are exact in double; u64 ones compared via key2 */
    uint64_t key2; /* u32 path: the 64-bit distance */
    uint32_t v;
} hnode;

typedef struct {
    hnode* a;
    uint64_t n, cap;
    int by_u64;
} heap_t;

static int hless(const heap_t* h, const hnode* x, const hnode* y) {
    return h->by_u64 ? x->key2 < y->key2 : x->key < y->key;
}

static void hpush(heap_t* h, hnode x) {
    uint64_t i;
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = (hnode*)realloc(h->a, sizeof(hnode) * h->cap);
    }
    i = h->n++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!hless(h, &x, &h->a[p])) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i] = x;
}

static hnode hpop(heap_t* h) {
    hnode top = h->a[0], x = h->a[--h->n];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        const hnode* best = &x;
        if (l < h->n && hless(h, &h->a[l], best)) { m = l; best = &h->a[l]; }
        if (r < h->n && hless(h, &h->a[r], best)) { m = r; best = &h->a[r]; }
        if (m == i) break;
        h->a[i] = h->a[m];
        i = m;
    }
    if (h->n) h->a[i] = x;
    return top;
}

/*
 * Single-source shortest paths.  dist_bits[v]: u32 distance, or the bits of
 * the f32 distance.  pred[v]: the smallest vertex id u with a tight edge
 * (u,v), i.e. d(u) + w(u,v) == d(v) (the canonical predecessor).
 */
int orc_dijkstra(uint32_t V, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* wbits, int wtype,
                 uint32_t s, uint32_t* dist_bits, uint32_t* pred) {
    heap_t h = {0};
    uint32_t u;
    int status = ORC_OK;
    if (s >= V) return ORC_EINVAL;
    h.by_u64 = (wtype == 0);
    if (wtype == 0) {
        uint64_t* d = (uint64_t*)malloc(sizeof(uint64_t) * V);
        for (u = 0; u < V; ++u) d[u] = UINT64_MAX;
        d[s] = 0;
        hpush(&h, (hnode){0.0, 0, s});
        while (h.n) {
            hnode x = hpop(&h);
            uint32_t e;
            if (x.key2 > d[x.v]) continue; /* stale entry */
            for (e = row_ptr[x.v]; e < row_ptr[x.v + 1]; ++e) {
                uint64_t c = d[x.v] + (uint64_t)wbits[e];
                if (c < d[col[e]]) {
                    d[col[e]] = c;
                    hpush(&h, (hnode){0.0, c, col[e]});
                }
            }
        }
        for (u = 0; u < V; ++u) {
            pred[u] = NONE;
            if (d[u] == UINT64_MAX) {
                dist_bits[u] = INF32;
            } else if (d[u] >= INF32) {
                dist_bits[u] = INF32; /* does not fit: reported unreachable */
                status = ORC_OVERFLOW;
            } else {
                dist_bits[u] = (uint32_t)d[u];
            }
        }
        for (u = 0; u < V; ++u) {
            uint32_t e;
            if (dist_bits[u] == INF32) continue;
            for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                uint32_t v = col[e];
                if (v == s || dist_bits[v] == INF32) continue;
                if ((uint64_t)dist_bits[u] + wbits[e] == (uint64_t)dist_bits[v] && u < pred[v]) pred[v] = u;
            }
        }
        free(d);
    } else {
        float* d = (float*)malloc(sizeof(float) * V);
        for (u = 0; u < V; ++u) d[u] = INFINITY;
        d[s] = 0.0f;
        hpush(&h, (hnode){0.0, 0, s});
        while (h.n) {
            hnode x = hpop(&h);
            uint32_t e;
            if ((float)x.key > d[x.v]) continue;
            for (e = row_ptr[x.v]; e < row_ptr[x.v + 1]; ++e) {
                volatile float c = d[x.v] + f32_of(wbits[e]); /* one float32 rounding */
                if (c < d[col[e]]) {
                    d[col[e]] = c;
                    hpush(&h, (hnode){(double)c, 0, col[e]});
                }
            }
        }
        for (u = 0; u < V; ++u) {
            pred[u] = NONE;
            if (isinf(d[u])) {
                dist_bits[u] = bits_of(INFINITY);
            } else {
                dist_bits[u] = bits_of(d[u]);
            }
        }
        for (u = 0; u < V; ++u) {
            uint32_t e;
            if (isinf(d[u])) continue;
            for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                uint32_t v = col[e];
                volatile float c;
                if (v == s || isinf(d[v])) continue;
                c = d[u] + f32_of(wbits[e]);
                if (c == d[v] && u < pred[v]) pred[v] = u;
            }
        }
        free(d);
    }
    free(h.a);
    return status;
}

/* Count of reached vertices v != s with more than one tight in-edge. */
uint64_t orc_tight_ties(uint32_t V, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* wbits,
                        int wtype, uint32_t s, const uint32_t* dist_bits) {
    uint32_t* cnt = (uint32_t*)calloc(V, sizeof(uint32_t));
    uint32_t u;
    uint64_t ties = 0;
    for (u = 0; u < V; ++u) {
        uint32_t e;
        if (wtype == 0 ? dist_bits[u] == INF32 : isinf(f32_of(dist_bits[u]))) continue;
        for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t v = col[e];
            if (v == s) continue;
            if (wtype == 0) {
                if (dist_bits[v] != INF32 && (uint64_t)dist_bits[u] + wbits[e] == dist_bits[v]) cnt[v]++;
            } else {
                volatile float c = f32_of(dist_bits[u]) + f32_of(wbits[e]);
                if (!isinf(f32_of(dist_bits[v])) && c == f32_of(dist_bits[v])) cnt[v]++;
            }
        }
    }
    for (u = 0; u < V; ++u) ties += cnt[u] > 1;
    free(cnt);
    return ties;
}

/* ----------------------------------------------------------------- Trishla */

static int64_t find_edge(const uint32_t* row_ptr, const uint32_t* col, uint32_t a, uint32_t b) {
    uint32_t lo = row_ptr[a], hi = row_ptr[a + 1];
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (col[mid] < b)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < row_ptr[a + 1] && col[lo] == b) ? (int64_t)lo : -1;
}

/* is w(u,vj) > w(u,vi) + w(vi,vj) ? (the test of Algorithm 1) */
static int dominated(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj, int wtype) {
    if (wtype == 0) return (uint64_t)w_uvj > (uint64_t)w_uvi + (uint64_t)w_vivj;
    {
        volatile float sum = f32_of(w_uvi) + f32_of(w_vivj);
        return f32_of(w_uvj) > sum;
    }
}

/*
 * Algorithm 1 on the rows u in [u_lo, u_hi).  For every u and every ordered
 * pair (v_i, v_j) of distinct out-neighbours of u such that (v_i, v_j) is an
 * edge -- and, in local mode (mode 0), v_i belongs to u's partition, so that
 * (v_i, v_j) is in that partition's edge set E_i -- the edge (u, v_j) is
 * deleted when w(u,v_j) > w(u,v_i) + w(v_i,v_j).  All tests use the unpruned
 * graph.  keep[e] = 0 for deleted edges (1 otherwise); witness[e] = the
 * smallest such v_i (NONE for kept edges).  P is the partition count.
 */
int orc_trishla(uint32_t V, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* wbits, int wtype,
                uint32_t P, int mode, uint32_t u_lo, uint32_t u_hi, uint8_t* keep, uint32_t* witness) {
    uint64_t B;
    uint32_t u;
    if (P == 0 || V == 0 || u_hi > V || u_lo > u_hi) return ORC_EINVAL;
    B = ((uint64_t)V + P - 1) / P;
    for (u = u_lo; u < u_hi; ++u) {
        uint32_t j;
        for (j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            uint32_t i;
            keep[j] = 1;
            witness[j] = NONE;
            for (i = row_ptr[u]; i < row_ptr[u + 1]; ++i) {
                uint32_t vi = col[i], vj = col[j];
                int64_t e2;
                if (i == j) continue;
                if (mode == 0 && (uint64_t)vi / B != (uint64_t)u / B) continue;
                e2 = find_edge(row_ptr, col, vi, vj);
                if (e2 < 0) continue;
                if (dominated(wbits[j], wbits[i], wbits[e2], wtype)) {
                    keep[j] = 0;
                    if (vi < witness[j]) witness[j] = vi;
                }
            }
        }
    }
    return ORC_OK;
}

/* ----------------------------------------------------------- tree gradient */

typedef struct {
    float d;
    uint32_t v;
} dv_t;

static int dv_desc(const void* pa, const void* pb) {
    const dv_t* a = (const dv_t*)pa;
    const dv_t* b = (const dv_t*)pb;
    if (a->d != b->d) return a->d > b->d ? -1 : 1;
    return a->v < b->v ? -1 : (a->v > b->v);
}

/*
 * grad[e] (float64, CSR edge order, accumulated over the S sources) of
 * L = sum_s sum_v g[s][v] * dist_s(v) with respect to w(e), given each
 * source's distances dist[s][V] (f32) and canonical predecessors pred[s][V].
 * Vertices are visited in decreasing distance; each reached v != source adds
 * its accumulated subtree sum acc[v] to the tree edge (pred(v), v) and to
 * acc[pred(v)].  Unreachable vertices contribute nothing.
 * Returns ORC_EINVAL if a predecessor edge is not in the graph.
 */
int orc_tree_grad(uint32_t V, const uint32_t* row_ptr, const uint32_t* col, uint32_t S, const float* dist,
                  const uint32_t* pred, const float* g, double* grad) {
    uint32_t s, e;
    double* acc = (double*)malloc(sizeof(double) * (V ? V : 1));
    dv_t* order = (dv_t*)malloc(sizeof(dv_t) * (V ? V : 1));
    for (e = 0; e < row_ptr[V]; ++e) grad[e] = 0.0;
    for (s = 0; s < S; ++s) {
        const float* d = dist + (uint64_t)s * V;
        const uint32_t* p = pred + (uint64_t)s * V;
        const float* gs = g + (uint64_t)s * V;
        uint32_t n = 0, v, k;
        for (v = 0; v < V; ++v) {
            acc[v] = (double)gs[v];
            if (!isinf(d[v])) {
                order[n].d = d[v];
                order[n].v = v;
                ++n;
            }
        }
        qsort(order, n, sizeof(dv_t), dv_desc);
        for (k = 0; k < n; ++k) {
            int64_t te;
            v = order[k].v;
            if (p[v] == NONE) continue; /* the source */
            te = find_edge(row_ptr, col, p[v], v);
            if (te < 0) {
                free(acc);
                free(order);
                return ORC_EINVAL;
            }
            grad[te] += acc[v];
            acc[p[v]] += acc[v];
        }
    }
    free(acc);
    free(order);
    return ORC_OK;
}
