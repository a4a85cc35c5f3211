// C ABI of libsssp (declared in include/sssp.h): argument checks, workspace
// layout, launch configuration and the batched CUDA-graph plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace sssp;

namespace {

constexpr uint32_t DEF_THREADS = 512;
constexpr uint32_t DEF_TILE = 1024;
constexpr uint64_t DEF_TIMEOUT_NS = 20ull * 1000 * 1000 * 1000;
constexpr uint32_t MAX_UNITS_PER_SOURCE = 65536;
// Default bucket widths: about 1/32 of the mean weight of the workloads this library
// is tuned on (uint32 U{1..255}: 4; float32 U[0.5,2): 1/16).  Measured on R-MAT scale 22:
// smaller widths scan fewer edges (closer to Dijkstra order), larger ones need fewer rounds.
constexpr uint32_t DEF_DELTA_U32 = 4;
constexpr float DEF_DELTA_F32 = 0.0625f;

struct Resolved {
    uint32_t threads, tile, split, bps;
    uint32_t delta_bits, policy, msg_buffer, hub_count, hub_delta_bits, hub_mid_bits;
    uint64_t timeout_ns;
    uint32_t flags;
    cudaEvent_t ev_begin, ev_end;
};

bool graph_ok(const sssp_graph* g) {
    if (!g || g->V == 0 || g->partitions == 0 || g->partitions > g->V) return false;
    if (!g->row_ptr || (g->E && (!g->col || !g->w))) return false;
    if (g->wtype != SSSP_W_U32 && g->wtype != SSSP_W_F32) return false;
    if ((g->ids == nullptr) != (g->slots == nullptr)) return false;
    return true;
}

uint32_t delta_bits_for(int wtype, double delta) {
    if (wtype == SSSP_W_F32) {
        float f = (delta > 0.0) ? (float)delta : DEF_DELTA_F32;
        uint32_t b;
        std::memcpy(&b, &f, 4);
        return b;
    }
    if (delta <= 0.0) return DEF_DELTA_U32;
    return (uint32_t)std::min(4294967294.0, std::max(1.0, std::floor(delta)));
}

// bucket width of hubs: the round's over 2^shift (at least one unit for uint32 distances)
uint32_t hub_delta_bits_for(int wtype, uint32_t delta_bits, int shift) {
    if (wtype == SSSP_W_F32) {
        float f;
        std::memcpy(&f, &delta_bits, 4);
        f = std::ldexp(f, -shift);
        uint32_t b;
        std::memcpy(&b, &f, 4);
        return b;
    }
    return std::max(1u, delta_bits >> shift);
}

bool resolve(const sssp_options* o, int wtype, Resolved* r) {
    sssp_options d{};
    if (!o) o = &d;
    r->threads = o->threads ? o->threads : DEF_THREADS;
    r->tile = o->tile ? o->tile : DEF_TILE;
    r->split = o->split ? o->split : 1u;
    r->bps = o->blocks_per_sm;
    r->delta_bits = delta_bits_for(wtype, o->delta);
    r->timeout_ns = o->timeout_ns ? o->timeout_ns : DEF_TIMEOUT_NS;
    r->flags = o->flags;
    r->policy = o->policy;
    r->msg_buffer = o->msg_buffer;
    r->hub_count = o->hub_count;
    r->hub_delta_bits = hub_delta_bits_for(wtype, r->delta_bits, 2);
    r->hub_mid_bits = hub_delta_bits_for(wtype, r->delta_bits, 1);
    r->ev_begin = static_cast<cudaEvent_t>(o->ev_relax_begin);
    r->ev_end = static_cast<cudaEvent_t>(o->ev_relax_end);
    if (r->threads < 128 || r->threads > 1024 || (r->threads % 32)) return false;
    if (r->tile < 32 || r->tile > 4096) return false;
    if (r->split > 1024) return false;
    if (r->policy > SSSP_POLICY_ALL) return false;
    if (r->msg_buffer > 32) return false;
    if (!(o->delta >= 0.0) || std::isinf(o->delta)) return false;
    return true;
}

// Workspace of sssp_solve: header | packed[S][V] | bitmap[S][words] | dirty[S*Q] | nfsplit[S*Q]
struct SolveWs {
    size_t off_packed, off_bitmap, off_dirty, off_nf, total;
    uint32_t words, B, Bq, Q;
};

SolveWs solve_layout(const sssp_graph* g, uint32_t S, uint32_t split) {
    SolveWs w{};
    w.words = (g->V + 31u) / 32u;
    w.B = (uint32_t)(((uint64_t)g->V + g->partitions - 1) / g->partitions);
    w.Bq = (w.B + split - 1u) / split;
    w.Q = g->partitions * split;
    size_t off = WS_HEADER_BYTES;
    w.off_packed = off;
    off += align_up(8ull * S * g->V, 256);
    w.off_bitmap = off;
    off += align_up(4ull * S * w.words, 256);
    w.off_dirty = off;
    off += align_up(4ull * S * w.Q, 256);
    w.off_nf = off;
    off += align_up(4ull * S * w.Q, 256);
    w.total = off;
    return w;
}

int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

const char* sssp_status_string(sssp_status s) {
    switch (s) {
        case SSSP_OK: return "ok";
        case SSSP_EINVAL: return "invalid argument";
        case SSSP_ENOMEM: return "workspace too small";
        case SSSP_ECUDA: return "CUDA runtime error";
        case SSSP_ETIMEOUT: return "device wait timed out";
        case SSSP_EOVERFLOW: return "uint32 distance overflow";
        case SSSP_EINTERNAL: return "internal error";
        case SSSP_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* sssp_version(void) { return "libsssp 0.1 sm_103a"; }

size_t sssp_build_csr_workspace_size(uint32_t V, uint64_t E_raw) { return csr_workspace_bytes(V, E_raw); }

sssp_status sssp_build_csr(uint32_t V, uint64_t E_raw, const uint32_t* src, const uint32_t* dst, const void* w,
                           int32_t wtype, uint32_t* row_ptr, uint32_t* col, void* w_out, uint32_t* eid,
                           uint32_t* E_out, void* ws, size_t ws_bytes, sssp_stream_t stream) {
    if (V == 0 || E_raw >= 0xFFFFFFFFull || !row_ptr || !E_out || !ws) return SSSP_EINVAL;
    if (E_raw && (!src || !dst || !w || !col || !w_out)) return SSSP_EINVAL;
    if (wtype != SSSP_W_U32 && wtype != SSSP_W_F32) return SSSP_EINVAL;
    return csr_build(V, E_raw, src, dst, static_cast<const uint32_t*>(w), wtype, row_ptr, col,
                     static_cast<uint32_t*>(w_out), eid, E_out, ws, ws_bytes, (cudaStream_t)stream);
}

size_t sssp_layout_workspace_size(const sssp_graph* g) {
    if (!graph_ok(g) || g->ids) return 0;
    return layout_workspace_bytes(g->V, g->E);
}

sssp_status sssp_layout(const sssp_graph* g, uint32_t* row_ptr_out, uint32_t* col_out, void* w_out,
                        uint32_t* emap_out, uint32_t* ids_out, uint32_t* slots_out, void* ws, size_t ws_bytes,
                        sssp_stream_t stream) {
    if (!graph_ok(g) || g->ids || !row_ptr_out || !ids_out || !slots_out || !ws || !aligned16(ws)) return SSSP_EINVAL;
    if (g->E && (!col_out || !w_out)) return SSSP_EINVAL;
    if (ws_bytes < layout_workspace_bytes(g->V, g->E)) return SSSP_ENOMEM;
    return layout_build(g, row_ptr_out, col_out, static_cast<uint32_t*>(w_out), emap_out, ids_out, slots_out, ws,
                        ws_bytes, (cudaStream_t)stream);
}

sssp_status sssp_partition(const sssp_graph* g, uint32_t* bounds, uint64_t* inter, sssp_stream_t stream) {
    if (!graph_ok(g) || !bounds) return SSSP_EINVAL;
    return partition_launch(g, bounds, inter, (cudaStream_t)stream) == cudaSuccess ? SSSP_OK : SSSP_ECUDA;
}

sssp_status sssp_prune(const sssp_graph* g, int32_t mode, uint8_t* keep, uint32_t* witness, sssp_stream_t stream) {
    if (!graph_ok(g) || (mode != 0 && mode != 1) || (g->E && !keep)) return SSSP_EINVAL;
    return prune_launch(g, mode, keep, witness, (cudaStream_t)stream) == cudaSuccess ? SSSP_OK : SSSP_ECUDA;
}

size_t sssp_compact_workspace_size(uint32_t V, uint32_t E) { return compact_workspace_bytes(V, E); }

sssp_status sssp_compact(const sssp_graph* g, const uint8_t* keep, uint32_t* row_ptr_out, uint32_t* col_out,
                         void* w_out, uint32_t* emap_out, uint32_t* E_out, void* ws, size_t ws_bytes,
                         sssp_stream_t stream) {
    if (!graph_ok(g) || !row_ptr_out || !E_out || !ws || (g->E && (!keep || !col_out || !w_out))) return SSSP_EINVAL;
    return compact_launch(g, keep, row_ptr_out, col_out, static_cast<uint32_t*>(w_out), emap_out, E_out, ws, ws_bytes,
                          (cudaStream_t)stream);
}

size_t sssp_solve_workspace_size(const sssp_graph* g, uint32_t S, const sssp_options* opt) {
    Resolved r;
    if (!graph_ok(g) || S == 0 || !resolve(opt, g->wtype, &r)) return 0;
    return solve_layout(g, S, r.split).total;
}

// sssp_solve (sources given) and sssp_update (warm: from the result in dist/pred)
static sssp_status solve_impl(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                              const sssp_options* opt, void* ws, size_t ws_bytes, sssp_stream_t stream,
                              const uint32_t* tails, uint32_t n_tails, bool warm, int prune_mode = -1,
                              uint8_t* keep = nullptr, uint32_t* witness = nullptr) {
    Resolved r;
    if (!graph_ok(g) || S == 0 || (!warm && !sources) || !dist || !ws || !resolve(opt, g->wtype, &r))
        return SSSP_EINVAL;
    if (!aligned16(ws) || r.threads > SOLVE_MAX_THREADS) return SSSP_EINVAL;
    const SolveWs L = solve_layout(g, S, r.split);
    if ((uint64_t)S * L.Q > 0xFFFFFFFFull / 2 || L.Q > MAX_UNITS_PER_SOURCE * 16u) return SSSP_EINVAL;
    if (ws_bytes < L.total) return SSSP_ENOMEM;
    const size_t smem = relax_smem_bytes(r.tile, L.Q, r.msg_buffer != 0);
    if (smem > 200 * 1024) return SSSP_EINVAL;
    const bool prune = prune_mode >= 0;
    int per_sm = 0;
    const uint32_t hubs = g->ids ? std::min(r.hub_count, L.B) : 0u;  // layout graphs only
    if (relax_max_blocks_per_sm(g->wtype, r.threads, r.tile, L.Q, &per_sm, prune, r.msg_buffer != 0, hubs != 0) !=
        cudaSuccess)
        return SSSP_ECUDA;
    if (per_sm <= 0) return SSSP_EUNSUPPORTED;
    if (r.bps) per_sm = std::min<int>(per_sm, (int)r.bps);
    const uint64_t U = (uint64_t)S * L.Q;
    SolveLaunch l{};
    l.row_ptr = g->row_ptr;
    l.col = g->col;
    l.w = static_cast<const uint32_t*>(g->w);
    l.wtype = g->wtype;
    l.V = g->V;
    l.ids = g->ids;
    l.slots = g->slots;
    l.S = S;
    l.sources = sources;
    l.B = L.B;
    l.Bq = L.Bq;
    l.split = r.split;
    l.Q = L.Q;
    l.words = L.words;
    char* base = static_cast<char*>(ws);
    l.hdr = reinterpret_cast<WsHeader*>(base);
    l.packed = reinterpret_cast<unsigned long long*>(base + L.off_packed);
    l.bitmap = reinterpret_cast<uint32_t*>(base + L.off_bitmap);
    l.dirty = reinterpret_cast<uint32_t*>(base + L.off_dirty);
    l.nfsplit = reinterpret_cast<uint32_t*>(base + L.off_nf);
    l.threads = r.threads;
    l.tile = r.tile;
    l.grid = (uint32_t)std::min<uint64_t>(U, (uint64_t)per_sm * sm_count());
    l.delta_bits = r.delta_bits;
    l.policy = r.policy;
    l.msg_buffer = r.msg_buffer;
    l.hub_count = hubs;
    l.hub_delta_bits = r.hub_delta_bits;
    l.hub_mid_bits = r.hub_mid_bits;
    l.timeout_ns = r.timeout_ns;
    l.hold_pending = (r.flags & SSSP_FLAG_TEST_HOLD_PENDING) ? 1u : 0u;
    l.ev_begin = r.ev_begin;
    l.ev_end = r.ev_end;
    l.dist = static_cast<uint32_t*>(dist);
    l.pred = pred;
    l.warm = warm ? 1u : 0u;
    l.warm_tails = tails;
    l.n_tails = n_tails;
    l.prune_on = prune ? 1u : 0u;
    if (prune) l.prune = trishla_job(g, prune_mode, keep, witness);
    return launch_solve(l, (cudaStream_t)stream) == cudaSuccess ? SSSP_OK : SSSP_ECUDA;
}

sssp_status sssp_solve(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                       const sssp_options* opt, void* ws, size_t ws_bytes, sssp_stream_t stream) {
    return solve_impl(g, sources, S, dist, pred, opt, ws, ws_bytes, stream, nullptr, 0, false);
}

sssp_status sssp_solve_prune(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                             int32_t mode, uint8_t* keep, uint32_t* witness, const sssp_options* opt, void* ws,
                             size_t ws_bytes, sssp_stream_t stream) {
    if ((mode != 0 && mode != 1) || (g && g->E && !keep)) return SSSP_EINVAL;
    return solve_impl(g, sources, S, dist, pred, opt, ws, ws_bytes, stream, nullptr, 0, false, mode, keep, witness);
}

sssp_status sssp_update(const sssp_graph* g, uint32_t S, void* dist, uint32_t* pred, const uint32_t* tails,
                        uint32_t n_tails, const sssp_options* opt, void* ws, size_t ws_bytes, sssp_stream_t stream) {
    if (!pred || (n_tails && !tails)) return SSSP_EINVAL;
    return solve_impl(g, nullptr, S, dist, pred, opt, ws, ws_bytes, stream, tails, n_tails, true);
}

sssp_status sssp_autotune(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                          void* ws, size_t ws_bytes, const sssp_options* base, uint32_t trials,
                          sssp_options* best, float* best_ms, sssp_stream_t stream) {
    if (!graph_ok(g) || S == 0 || !sources || !dist || !ws || !best) return SSSP_EINVAL;
    sssp_options b{};
    if (base) b = *base;
    b.ev_relax_begin = b.ev_relax_end = nullptr;
    Resolved r;
    if (!resolve(&b, g->wtype, &r)) return SSSP_EINVAL;
    b.threads = r.threads;  // report explicit values, not "default" zeros
    b.tile = r.tile;
    b.split = r.split;
    if (trials == 0) trials = 1;
    cudaStream_t st = (cudaStream_t)stream;
    // mean of a sample of the weights sets the scale of the bucket-width candidates
    double mean = 1.0;
    if (g->E) {
        const uint32_t n = std::min<uint32_t>(g->E, 65536);
        std::vector<uint32_t> h(n);
        if (cudaMemcpyAsync(h.data(), g->w, 4ull * n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SSSP_ECUDA;
        double sum = 0;
        for (uint32_t x : h) {
            if (g->wtype == SSSP_W_F32) {
                float f;
                std::memcpy(&f, &x, 4);
                sum += f;
            } else {
                sum += x;
            }
        }
        mean = sum / n;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SSSP_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SSSP_ECUDA;
    }
    // time one candidate: warm-up, then `trials` runs; +inf if it fails
    auto run = [&](const sssp_options& o) -> float {
        if (sssp_solve_workspace_size(g, S, &o) > ws_bytes || sssp_solve_workspace_size(g, S, &o) == 0)
            return INFINITY;
        if (sssp_solve(g, sources, S, dist, pred, &o, ws, ws_bytes, stream) != SSSP_OK) return INFINITY;
        if (sssp_workspace_status(ws, stream, nullptr) != SSSP_OK) return INFINITY;
        cudaEventRecord(e0, st);
        for (uint32_t t = 0; t < trials; ++t)
            if (sssp_solve(g, sources, S, dist, pred, &o, ws, ws_bytes, stream) != SSSP_OK) return INFINITY;
        cudaEventRecord(e1, st);
        if (sssp_workspace_status(ws, stream, nullptr) != SSSP_OK) return INFINITY;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return INFINITY;
        return ms / (float)trials;
    };
    sssp_options cur = b;
    float cur_ms = INFINITY;
    const double factors[] = {1.0 / 64, 1.0 / 32, 1.0 / 16, 1.0 / 8, 1.0 / 4, 1.0 / 2, 1.0, 2.0, 4.0};
    for (uint32_t pol : {(uint32_t)SSSP_POLICY_RELATIVE, (uint32_t)SSSP_POLICY_FIXED, (uint32_t)SSSP_POLICY_NEAR_FAR,
                         (uint32_t)SSSP_POLICY_ALL}) {
        for (double f : factors) {
            sssp_options o = b;
            o.policy = pol;
            o.delta = g->wtype == SSSP_W_F32 ? mean * f : std::max(1.0, std::floor(mean * f));
            const float ms = run(o);
            if (ms < cur_ms) {
                cur_ms = ms;
                cur = o;
            }
            if (pol == SSSP_POLICY_ALL) break;  // delta unused
        }
    }
    // refine the bucket width between the coarse steps
    const double coarse = cur.delta;
    for (double f : {0.75, 1.5}) {
        sssp_options o = cur;
        o.delta = g->wtype == SSSP_W_F32 ? coarse * f : std::max(1.0, std::floor(coarse * f));
        if (o.delta == coarse) continue;
        const float ms = run(o);
        if (ms < cur_ms) {
            cur_ms = ms;
            cur = o;
        }
    }
    // on a layout graph: hubs (the highest-degree stored vertices of each partition) on a quarter of
    // the width, and the other vertices on a wider bucket than the best without hubs
    if (g->ids) {
        const sssp_options nohub = cur;
        for (uint32_t pol : {(uint32_t)SSSP_POLICY_RELATIVE, (uint32_t)SSSP_POLICY_FIXED, (uint32_t)SSSP_POLICY_NEAR_FAR}) {
            for (uint32_t hubs : {256u, 512u, 1024u}) {
                for (double f : {1.0, 1.5, 2.0, 3.0}) {
                    sssp_options o = nohub;
                    o.policy = pol;
                    o.hub_count = hubs;
                    o.delta = g->wtype == SSSP_W_F32 ? nohub.delta * f : std::max(1.0, std::floor(nohub.delta * f));
                    const float ms = run(o);
                    if (ms < cur_ms) {
                        cur_ms = ms;
                        cur = o;
                    }
                }
            }
        }
    }
    for (uint32_t tile : {1024u, 2048u, 4096u}) {
        sssp_options o = cur;
        o.tile = tile;
        const float ms = run(o);
        if (ms < cur_ms) {
            cur_ms = ms;
            cur = o;
        }
    }
    for (uint32_t split : {1u, 2u, 4u}) {
        sssp_options o = cur;
        o.split = split;
        const float ms = run(o);
        if (ms < cur_ms) {
            cur_ms = ms;
            cur = o;
        }
    }
    // the tile again at the chosen split (the best tile depends on it: the 4096-square grid takes
    // 4096 at split 1 but 2048 at split 4)
    if (cur.split != 1) {
        for (uint32_t tile : {1024u, 2048u, 4096u}) {
            if (tile == cur.tile) continue;
            sssp_options o = cur;
            o.tile = tile;
            const float ms = run(o);
            if (ms < cur_ms) {
                cur_ms = ms;
                cur = o;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!(cur_ms < INFINITY)) return SSSP_EINTERNAL;  // no candidate ran
    // leave a valid solve of the chosen schedule in dist/pred
    if (sssp_solve(g, sources, S, dist, pred, &cur, ws, ws_bytes, stream) != SSSP_OK) return SSSP_ECUDA;
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return sssp_workspace_status(ws, stream, nullptr);
}

sssp_status sssp_workspace_status(const void* ws, sssp_stream_t stream, sssp_stats* stats) {
    if (!ws) return SSSP_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SSSP_ECUDA;
    WsHeader h;
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return SSSP_ECUDA;
    if (stats) {
        static_assert(sizeof(sssp_stats) == 9 * sizeof(uint64_t), "stats layout");
        std::memcpy(stats, h.stats, sizeof(sssp_stats));
    }
    return (sssp_status)h.status;
}

// ------------------------------------------------------------------ sharding

sssp_status sssp_shard_problems(uint32_t n_problems, const uint64_t* cost, uint32_t n_ranks, uint32_t* rank_of,
                                uint64_t* load) {
    if (n_ranks == 0 || (n_problems && (!cost || !rank_of))) return SSSP_EINVAL;
    std::vector<uint32_t> order(n_problems);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
    // min-heap of (load, rank): the least loaded rank, lowest rank on ties
    std::vector<std::pair<uint64_t, uint32_t>> heap(n_ranks);
    for (uint32_t r = 0; r < n_ranks; ++r) heap[r] = {0ull, r};
    auto greater = [](const std::pair<uint64_t, uint32_t>& x, const std::pair<uint64_t, uint32_t>& y) {
        return x > y;
    };
    std::make_heap(heap.begin(), heap.end(), greater);
    for (uint32_t i : order) {
        std::pop_heap(heap.begin(), heap.end(), greater);
        rank_of[i] = heap.back().second;
        heap.back().first += cost[i];
        std::push_heap(heap.begin(), heap.end(), greater);
    }
    if (load)
        for (const auto& h : heap) load[h.second] = h.first;
    return SSSP_OK;
}

// ------------------------------------------------------------------ batched

namespace {

struct BatchTables {
    std::vector<BatchProblem> probs;  // in processing order
    uint64_t total_out = 0, total_words = 0;
};

bool build_tables(const sssp_batch* b, BatchTables* t) {
    if (!b || !b->graphs || !b->prob_graph || !b->prob_source || !b->row_ptr || !b->dist) return false;
    if (b->wtype != SSSP_W_U32 && b->wtype != SSSP_W_F32) return false;
    if (b->n_problems == 0 || b->n_graphs == 0) return false;
    t->probs.resize(b->n_problems);
    uint64_t out = 0;
    for (uint32_t i = 0; i < b->n_problems; ++i) {
        const uint32_t gi = b->prob_graph[i];
        if (gi >= b->n_graphs) return false;
        const sssp_batch_graph& G = b->graphs[gi];
        if (G.V == 0 || b->prob_source[i] >= G.V) return false;
        BatchProblem& p = t->probs[i];
        p.row_off = G.row_off;
        p.edge_off = G.edge_off;
        p.out_off = out;
        // disjoint inbox words: floor((out + 31 i) / 32) .. + ceil(V / 32)
        p.bm_off = (out + 31ull * i) / 32ull;
        p.V = G.V;
        p.src = b->prob_source[i];
        p.E = G.E;
        p.pad = 0;
        out += G.V;
    }
    t->total_out = out;
    t->total_words = (out + 31ull * b->n_problems) / 32ull + 1;
    // largest graphs first (longest-processing-time order), stable
    std::stable_sort(t->probs.begin(), t->probs.end(),
                     [](const BatchProblem& x, const BatchProblem& y) { return x.E > y.E; });
    return true;
}

struct BatchWs {
    size_t off_probs, off_packed, off_bitmap, total;
};

BatchWs batch_layout(uint32_t n_problems, uint64_t total_out, uint64_t total_words) {
    BatchWs w{};
    size_t off = WS_HEADER_BYTES;
    w.off_probs = off;
    off += align_up(sizeof(BatchProblem) * (size_t)n_problems, 256);
    w.off_packed = off;
    off += align_up(8ull * total_out, 256);
    w.off_bitmap = off;
    off += align_up(4ull * total_words * batched_bitmaps(), 256);
    w.total = off;
    return w;
}

sssp_status prepare_batch(const sssp_batch* b, const sssp_options* opt, void* ws, size_t ws_bytes,
                          cudaStream_t st, BatchLaunch* l) {
    Resolved r;
    BatchTables t;
    if (!ws || !aligned16(ws) || !resolve(opt, b ? b->wtype : 0, &r) || !build_tables(b, &t)) return SSSP_EINVAL;
    if (r.threads > BATCH_MAX_THREADS) return SSSP_EINVAL;
    const BatchWs L = batch_layout(b->n_problems, t.total_out, t.total_words);
    if (ws_bytes < L.total) return SSSP_ENOMEM;
    char* base = static_cast<char*>(ws);
    if (cudaMemcpyAsync(base + L.off_probs, t.probs.data(), sizeof(BatchProblem) * t.probs.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SSSP_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SSSP_ECUDA;
    int per_sm = 0;
    if (batched_max_blocks_per_sm(b->wtype, r.threads, r.tile, &per_sm) != cudaSuccess) return SSSP_ECUDA;
    if (per_sm <= 0) return SSSP_EUNSUPPORTED;
    if (r.bps) per_sm = std::min<int>(per_sm, (int)r.bps);
    l->row_ptr = b->row_ptr;
    l->col = b->col;
    l->w = static_cast<const uint32_t*>(b->w);
    l->wtype = b->wtype;
    l->n_problems = b->n_problems;
    l->probs = reinterpret_cast<const BatchProblem*>(base + L.off_probs);
    l->hdr = reinterpret_cast<WsHeader*>(base);
    l->packed = reinterpret_cast<unsigned long long*>(base + L.off_packed);
    l->bitmap = reinterpret_cast<uint32_t*>(base + L.off_bitmap);
    l->threads = r.threads;
    l->tile = r.tile;
    l->grid = (uint32_t)std::min<uint64_t>(b->n_problems, (uint64_t)per_sm * sm_count());
    l->delta_bits = r.delta_bits;
    l->timeout_ns = r.timeout_ns;
    l->dist = static_cast<uint32_t*>(b->dist);
    l->pred = b->pred;
    l->ev_begin = r.ev_begin;
    l->ev_end = r.ev_end;
    return SSSP_OK;
}

}  // namespace

size_t sssp_batch_workspace_size(const sssp_batch* b, const sssp_options* opt) {
    Resolved r;
    BatchTables t;
    if (!resolve(opt, b ? b->wtype : 0, &r) || !build_tables(b, &t)) return 0;
    return batch_layout(b->n_problems, t.total_out, t.total_words).total;
}

sssp_status sssp_solve_batched(const sssp_batch* b, const sssp_options* opt, void* ws, size_t ws_bytes,
                               sssp_stream_t stream) {
    BatchLaunch l{};
    const sssp_status st = prepare_batch(b, opt, ws, ws_bytes, (cudaStream_t)stream, &l);
    if (st != SSSP_OK) return st;
    return launch_batched(l, (cudaStream_t)stream) == cudaSuccess ? SSSP_OK : SSSP_ECUDA;
}

struct sssp_batch_plan {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

sssp_status sssp_batch_plan_create(const sssp_batch* b, const sssp_options* opt, void* ws, size_t ws_bytes,
                                   sssp_stream_t stream, sssp_batch_plan** plan) {
    if (!plan) return SSSP_EINVAL;
    *plan = nullptr;
    BatchLaunch l{};
    cudaStream_t st = (cudaStream_t)stream;
    sssp_status s = prepare_batch(b, opt, ws, ws_bytes, st, &l);
    if (s != SSSP_OK) return s;
    // capture on a private stream so that the caller's stream may be the legacy default stream
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return SSSP_ECUDA;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    l.ev_begin = l.ev_end = nullptr;  // timing events are for direct launches only
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const cudaError_t le = launch_batched(l, cap);
        const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        ok = le == cudaSuccess && ce == cudaSuccess && graph;
    }
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaStreamDestroy(cap);
    if (!ok) {
        if (graph) cudaGraphDestroy(graph);
        return SSSP_ECUDA;
    }
    sssp_batch_plan* p = new sssp_batch_plan;
    p->graph = graph;
    p->exec = exec;
    *plan = p;
    return SSSP_OK;
}

sssp_status sssp_batch_plan_launch(sssp_batch_plan* plan, sssp_stream_t stream) {
    if (!plan) return SSSP_EINVAL;
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? SSSP_OK : SSSP_ECUDA;
}

void sssp_batch_plan_destroy(sssp_batch_plan* plan) {
    if (!plan) return;
    cudaGraphExecDestroy(plan->exec);
    cudaGraphDestroy(plan->graph);
    delete plan;
}

// ----------------------------------------------------------------- backward

size_t sssp_backward_workspace_size(uint32_t V, uint32_t E, uint32_t S) { return backward_workspace_bytes(V, E, S); }

sssp_status sssp_backward(const sssp_graph* g, uint32_t S, const uint32_t* pred, const float* grad_dist,
                          float* grad_w, void* ws, size_t ws_bytes, sssp_stream_t stream) {
    if (!graph_ok(g) || g->ids || S == 0 || !pred || !grad_dist || (g->E && !grad_w) || !ws) return SSSP_EINVAL;
    if (ws_bytes < backward_workspace_bytes(g->V, g->E, S)) return SSSP_ENOMEM;
    return backward_launch(g, S, pred, grad_dist, grad_w, ws, (cudaStream_t)stream) == cudaSuccess ? SSSP_OK
                                                                                                  : SSSP_ECUDA;
}

}  // extern "C"
