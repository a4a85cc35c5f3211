// K1 CSR builder, K2 block partitioner, edge compaction.
//
// K1 turns a raw edge list into the canonical adjacency (Sec. III.A's Padj
// for all partitions at once): keys (tail, head) are radix-sorted with their
// input index (a stable sort, so equal keys keep input order), runs of equal
// keys become one edge whose weight is the run's minimum (lowest input index
// on ties, via a 64-bit atomicMin on (weight bits << 32 | index)), and
// row_ptr is filled from the run boundaries.  Self-loops and bad ids sort to
// the end behind a sentinel key and are dropped.  The radix sort and the
// prefix sums are this library's own (sort.cu).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sssp {
namespace {

__host__ __device__ inline uint32_t bits_for(unsigned long long x) {
    uint32_t b = 0;
    while (b < 64 && (x >> b) != 0ull) ++b;
    return b;
}

struct CsrWs {
    WsHeader* hdr;
    unsigned long long *keys_in, *keys_out;
    uint32_t *vals_in, *vals_out;
    uint32_t* runinc;             // [E_raw] inclusive run index
    unsigned long long* runbest;  // [E_raw] (weight bits << 32 | input index)
    void* tmp;                    // sort and scan temporaries
    size_t total;
};

CsrWs carve_csr(void* ws, uint32_t V, uint64_t n) {
    (void)V;
    CsrWs c{};
    char* p = static_cast<char*>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = p ? p + off : nullptr;
        off += align_up(bytes, 256);
        return r;
    };
    c.hdr = reinterpret_cast<WsHeader*>(take(WS_HEADER_BYTES));
    c.keys_in = reinterpret_cast<unsigned long long*>(take(8 * n));
    c.keys_out = reinterpret_cast<unsigned long long*>(take(8 * n));
    c.vals_in = reinterpret_cast<uint32_t*>(take(4 * n));
    c.vals_out = reinterpret_cast<uint32_t*>(take(4 * n));
    c.runinc = reinterpret_cast<uint32_t*>(take(4 * n));
    c.runbest = reinterpret_cast<unsigned long long*>(take(8 * n));
    c.tmp = take(std::max(sort_temp_bytes(n), scan_temp_bytes(n)));
    c.total = off;
    return c;
}

template <class W>
__global__ void k_make_keys(uint32_t V, uint64_t n, const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                            const uint32_t* __restrict__ w, unsigned long long* keys, uint32_t* vals, WsHeader* hdr) {
    const unsigned long long sentinel = (unsigned long long)V * V;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = src[i], d = dst[i];
        unsigned long long k = sentinel;
        if (s >= V || d >= V || !W::weight_ok(w[i]))
            bad = true;
        else if (s != d)
            k = (unsigned long long)s * V + d;
        keys[i] = k;
        vals[i] = (uint32_t)i;
    }
    if (bad) set_status(hdr, SSSP_EINVAL);
}

// run head flag: first element of a run of equal valid keys
__global__ void k_heads(uint64_t n, unsigned long long sentinel, const unsigned long long* __restrict__ keys,
                        uint32_t* heads) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        heads[i] = (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
    }
}

__global__ void k_run_min(uint64_t n, unsigned long long sentinel, const unsigned long long* __restrict__ keys,
                          const uint32_t* __restrict__ vals, const uint32_t* __restrict__ w,
                          const uint32_t* __restrict__ runinc, unsigned long long* runbest) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (keys[i] == sentinel) continue;
        const uint32_t id = vals[i];
        atomicMin(&runbest[runinc[i] - 1u], ((unsigned long long)w[id] << 32) | id);
    }
}

// one thread per run head: emit the edge and the row_ptr entries up to its tail
__global__ void k_emit(uint32_t V, uint64_t n, unsigned long long sentinel, const unsigned long long* __restrict__ keys,
                       const uint32_t* __restrict__ runinc, const unsigned long long* __restrict__ runbest,
                       uint32_t* row_ptr, uint32_t* col, uint32_t* w_out, uint32_t* eid, uint32_t* E_out) {
    const uint32_t R = n ? runinc[n - 1] : 0u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        if (k == sentinel || (i > 0 && keys[i - 1] == k)) continue;
        const uint32_t r = runinc[i] - 1u;
        const uint32_t s = (uint32_t)(k / V), d = (uint32_t)(k % V);
        const unsigned long long best = runbest[r];
        col[r] = d;
        w_out[r] = (uint32_t)(best >> 32);
        if (eid) eid[r] = (uint32_t)best;
        // rows (s_prev, s] start at r
        const uint32_t s_prev = (r == 0) ? 0u : (uint32_t)(keys[i - 1] / V) + 1u;
        for (uint32_t u = (r == 0 ? 0u : s_prev); u <= s; ++u) row_ptr[u] = r;
        if (r + 1u == R)
            for (uint32_t u = s + 1u; u <= V; ++u) row_ptr[u] = R;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *E_out = R;
        if (R == 0)
            for (uint32_t u = 0; u <= V; ++u) row_ptr[u] = 0;
    }
}

// Block partition bounds and inter-edge counts.  A block takes a contiguous chunk of
// vertices: threads count the edges of low-degree vertices themselves; vertices of degree
// above PART_HUB are queued in shared memory and counted by the whole block together, so
// hubs do not serialise one thread.  Counts are summed per warp for lanes that share a
// partition before the atomic.
constexpr uint32_t PART_HUB = 256;
constexpr uint32_t PART_CHUNK = 4096;

// called by all 32 lanes of a warp: lanes that share pu add their counts with one atomic
__device__ __forceinline__ void add_inter(unsigned long long* inter, uint32_t pu, uint32_t c) {
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, pu);
    const uint32_t sum = __reduce_add_sync(peers, c);
    if ((__ffs(peers) - 1u) == (threadIdx.x & 31u) && sum) atomicAdd(&inter[pu], (unsigned long long)sum);
}

__global__ void k_partition(uint32_t V, uint32_t P, unsigned long long B, const uint32_t* __restrict__ row_ptr,
                            const uint32_t* __restrict__ col, uint32_t* bounds, unsigned long long* inter) {
    __shared__ uint32_t hubs[PART_CHUNK];
    __shared__ uint32_t nhub;
    __shared__ unsigned long long hub_cnt;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t p = gtid; p <= P; p += gridDim.x * blockDim.x)
        bounds[p] = (uint32_t)((unsigned long long)p * B < V ? (unsigned long long)p * B : V);
    if (!inter) return;
    for (uint32_t c0 = blockIdx.x * PART_CHUNK; c0 < V; c0 += gridDim.x * PART_CHUNK) {
        const uint32_t c1 = min(c0 + PART_CHUNK, V);
        if (threadIdx.x == 0) nhub = 0;
        __syncthreads();
        for (uint32_t base = c0; base < c1; base += blockDim.x) {  // same trip count for every thread
            const uint32_t u = base + threadIdx.x;
            uint32_t cnt = 0, pu = 0;
            if (u < c1) {
                pu = (uint32_t)(u / B);
                const uint32_t e0 = row_ptr[u], e1 = row_ptr[u + 1];
                if (e1 - e0 > PART_HUB) {
                    hubs[atomicAdd(&nhub, 1u)] = u;
                } else {
                    for (uint32_t e = e0; e < e1; ++e) cnt += (uint32_t)(col[e] / B) != pu;
                }
            }
            add_inter(inter, pu, cnt);
        }
        __syncthreads();
        for (uint32_t h = 0; h < nhub; ++h) {
            const uint32_t u = hubs[h];
            const uint32_t pu = (uint32_t)(u / B);
            if (threadIdx.x == 0) hub_cnt = 0;
            __syncthreads();
            unsigned long long cnt = 0;
            for (uint32_t e = row_ptr[u] + threadIdx.x; e < row_ptr[u + 1]; e += blockDim.x)
                cnt += (uint32_t)(col[e] / B) != pu;
            for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
            if ((threadIdx.x & 31u) == 0 && cnt) atomicAdd(&hub_cnt, cnt);
            __syncthreads();
            if (threadIdx.x == 0 && hub_cnt) atomicAdd(&inter[pu], hub_cnt);
        }
        __syncthreads();
    }
}

__global__ void k_keep_u32(uint32_t E, const uint8_t* __restrict__ keep, uint32_t* out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < E; i += gridDim.x * blockDim.x)
        out[i] = keep[i] ? 1u : 0u;
}

// pos = inclusive scan of keep
__global__ void k_compact(uint32_t V, uint32_t E, const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                          const uint32_t* __restrict__ w, const uint8_t* __restrict__ keep,
                          const uint32_t* __restrict__ pos, uint32_t* row_ptr_out, uint32_t* col_out,
                          uint32_t* w_out, uint32_t* emap, uint32_t* E_out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t i = gtid; i < E; i += stride) {
        if (!keep[i]) continue;
        const uint32_t j = pos[i] - 1u;
        col_out[j] = col[i];
        w_out[j] = w[i];
        if (emap) emap[j] = i;
    }
    for (uint32_t u = gtid; u <= V; u += stride) {
        const uint32_t r = row_ptr[u];
        row_ptr_out[u] = r == 0 ? 0u : pos[r - 1];
    }
    if (gtid == 0) *E_out = E ? pos[E - 1] : 0u;
}

// ---- locality layout: renumber vertices inside each block partition by degree

__global__ void k_lay_deg(uint32_t V, const uint32_t* __restrict__ row_ptr, uint32_t* deg) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
        deg[v] = row_ptr[v + 1] - row_ptr[v];
}

__global__ void k_lay_indeg(uint32_t V, uint32_t E, const uint32_t* __restrict__ col, uint32_t* deg) {
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const uint32_t v = col[e];
        if (v < V) atomicAdd(&deg[v], 1u);
    }
}

// key = (partition << 32) | ~degree: an ascending stable sort gives partitions in
// order, each by degree descending, ties by id ascending (the values start in id order)
__global__ void k_lay_keys(uint32_t V, unsigned long long B, const uint32_t* __restrict__ deg,
                           unsigned long long* keys, uint32_t* vals) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        keys[v] = ((unsigned long long)(v / B) << 32) | (0xFFFFFFFFu - deg[v]);
        vals[v] = v;
    }
}

__global__ void k_lay_slots(uint32_t V, const uint32_t* __restrict__ order, uint32_t* ids, uint32_t* slots) {
    for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < V; n += gridDim.x * blockDim.x) {
        const uint32_t v = order[n];
        ids[n] = v;
        slots[v] = n;
    }
}

// one warp per stored row: the edge list in the new numbering, in the old edge order
__global__ void k_lay_coo(uint32_t V, const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                          const uint32_t* __restrict__ slots, uint32_t* src, uint32_t* dst) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < V; u += warps) {
        const uint32_t beg = row_ptr[u], end = row_ptr[u + 1], su = slots[u];
        for (uint32_t e = beg + lane; e < end; e += 32u) {
            src[e] = su;
            const uint32_t v = col[e];
            dst[e] = v < V ? slots[v] : 0xFFFFFFFFu;  // a bad head stays bad: the CSR builder reports it
        }
    }
}

unsigned grid_for(uint64_t n, unsigned threads = 256) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 16));
}

}  // namespace

size_t csr_workspace_bytes(uint32_t V, uint64_t E_raw) { return carve_csr(nullptr, V, E_raw).total; }

#define CK(x)                                        \
    do {                                             \
        if ((x) != cudaSuccess) return SSSP_ECUDA;   \
    } while (0)

sssp_status csr_build(uint32_t V, uint64_t n, const uint32_t* src, const uint32_t* dst, const uint32_t* w, int wtype,
                      uint32_t* row_ptr, uint32_t* col, uint32_t* w_out, uint32_t* eid, uint32_t* E_out, void* ws,
                      size_t ws_bytes, cudaStream_t st) {
    CsrWs c = carve_csr(ws, V, n);
    if (ws_bytes < c.total) return SSSP_ENOMEM;
    const unsigned long long sentinel = (unsigned long long)V * V;
    const int end_bit = (int)bits_for(sentinel);
    CK(cudaMemsetAsync(c.hdr, 0, WS_HEADER_BYTES, st));
    CK(cudaMemsetAsync(row_ptr, 0, sizeof(uint32_t) * ((size_t)V + 1), st));
    CK(cudaMemsetAsync(E_out, 0, sizeof(uint32_t), st));
    if (n == 0) return SSSP_OK;
    const unsigned g = grid_for(n);
    if (wtype == SSSP_W_F32)
        k_make_keys<WF32><<<g, 256, 0, st>>>(V, n, src, dst, w, c.keys_in, c.vals_in, c.hdr);
    else
        k_make_keys<WU32><<<g, 256, 0, st>>>(V, n, src, dst, w, c.keys_in, c.vals_in, c.hdr);
    CK(cudaGetLastError());
    bool second = false;
    CK(sort_pairs_u64(c.tmp, c.keys_in, c.keys_out, c.vals_in, c.vals_out, n, end_bit, st, &second));
    const unsigned long long* sk = second ? c.keys_out : c.keys_in;  // sorted pairs
    const uint32_t* sv = second ? c.vals_out : c.vals_in;
    uint32_t* heads = second ? c.vals_in : c.vals_out;  // the other value buffer: head flags
    k_heads<<<g, 256, 0, st>>>(n, sentinel, sk, heads);
    CK(cudaGetLastError());
    CK(inclusive_scan_u32(c.tmp, heads, c.runinc, n, st));
    CK(cudaMemsetAsync(c.runbest, 0xFF, 8 * n, st));
    k_run_min<<<g, 256, 0, st>>>(n, sentinel, sk, sv, w, c.runinc, c.runbest);
    CK(cudaGetLastError());
    k_emit<<<g, 256, 0, st>>>(V, n, sentinel, sk, c.runinc, c.runbest, row_ptr, col, w_out, eid, E_out);
    CK(cudaGetLastError());
    return SSSP_OK;
}

cudaError_t partition_launch(const sssp_graph* g, uint32_t* bounds, uint64_t* inter, cudaStream_t st) {
    const unsigned long long B = ((unsigned long long)g->V + g->partitions - 1) / g->partitions;
    cudaError_t e;
    if (inter && (e = cudaMemsetAsync(inter, 0, sizeof(uint64_t) * g->partitions, st)) != cudaSuccess) return e;
    const uint64_t chunks = ((uint64_t)g->V + PART_CHUNK - 1) / PART_CHUNK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(chunks, (uint64_t)sms * 8));
    k_partition<<<blocks, 256, 0, st>>>(g->V, g->partitions, B, g->row_ptr, g->col, bounds,
                                        reinterpret_cast<unsigned long long*>(inter));
    return cudaGetLastError();
}

namespace {
struct LayoutWs {
    size_t off_deg, off_kin, off_kout, off_vin, off_vout, off_tmp, off_src, off_dst, off_eout, total;
    size_t csr_bytes, tmp_bytes;
};

LayoutWs layout_ws(uint32_t V, uint32_t E) {
    LayoutWs w{};
    w.csr_bytes = csr_workspace_bytes(V, E);
    w.tmp_bytes = sort_temp_bytes(V);
    size_t off = align_up(w.csr_bytes, 256);  // the CSR builder's workspace first: its header is the status word
    auto take = [&](size_t bytes) {
        const size_t r = off;
        off += align_up(std::max<size_t>(bytes, 4), 256);
        return r;
    };
    w.off_deg = take(4ull * V);
    w.off_kin = take(8ull * V);
    w.off_kout = take(8ull * V);
    w.off_vin = take(4ull * V);
    w.off_vout = take(4ull * V);
    w.off_tmp = take(w.tmp_bytes);
    w.off_src = take(4ull * E);
    w.off_dst = take(4ull * E);
    w.off_eout = take(4);
    w.total = off;
    return w;
}
}  // namespace

size_t layout_workspace_bytes(uint32_t V, uint32_t E) { return layout_ws(V, E).total; }

sssp_status layout_build(const sssp_graph* g, uint32_t* row_ptr_out, uint32_t* col_out, uint32_t* w_out,
                         uint32_t* emap_out, uint32_t* ids_out, uint32_t* slots_out, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
    const LayoutWs L = layout_ws(g->V, g->E);
    if (ws_bytes < L.total) return SSSP_ENOMEM;
    char* p = static_cast<char*>(ws);
    uint32_t* deg = reinterpret_cast<uint32_t*>(p + L.off_deg);
    unsigned long long* kin = reinterpret_cast<unsigned long long*>(p + L.off_kin);
    unsigned long long* kout = reinterpret_cast<unsigned long long*>(p + L.off_kout);
    uint32_t* vin = reinterpret_cast<uint32_t*>(p + L.off_vin);
    uint32_t* vout = reinterpret_cast<uint32_t*>(p + L.off_vout);
    uint32_t* src = reinterpret_cast<uint32_t*>(p + L.off_src);
    uint32_t* dst = reinterpret_cast<uint32_t*>(p + L.off_dst);
    uint32_t* eout = reinterpret_cast<uint32_t*>(p + L.off_eout);
    const unsigned long long B = ((unsigned long long)g->V + g->partitions - 1) / g->partitions;
    const unsigned gv = grid_for(g->V), ge = grid_for(std::max<uint32_t>(g->E, 1));
    k_lay_deg<<<gv, 256, 0, st>>>(g->V, g->row_ptr, deg);
    CK(cudaGetLastError());
    if (g->E) {
        k_lay_indeg<<<ge, 256, 0, st>>>(g->V, g->E, g->col, deg);
        CK(cudaGetLastError());
    }
    k_lay_keys<<<gv, 256, 0, st>>>(g->V, B, deg, kin, vin);
    CK(cudaGetLastError());
    bool second = false;
    CK(sort_pairs_u64(p + L.off_tmp, kin, kout, vin, vout, g->V, 32 + (int)bits_for(g->partitions - 1u), st, &second));
    k_lay_slots<<<gv, 256, 0, st>>>(g->V, second ? vout : vin, ids_out, slots_out);
    CK(cudaGetLastError());
    if (g->E) {
        k_lay_coo<<<grid_for((uint64_t)g->V * 32), 256, 0, st>>>(g->V, g->row_ptr, g->col, slots_out, src, dst);
        CK(cudaGetLastError());
    }
    // the renumbered edge list through the CSR builder: rows sorted by new head id, and
    // its input-index output maps each stored edge back to its index in g
    return csr_build(g->V, g->E, src, dst, static_cast<const uint32_t*>(g->w), g->wtype, row_ptr_out, col_out, w_out,
                     emap_out, eout, ws, L.csr_bytes, st);
}

size_t compact_workspace_bytes(uint32_t V, uint32_t E) {
    (void)V;
    return WS_HEADER_BYTES + 2 * align_up(4ull * std::max<uint32_t>(E, 1), 256) + align_up(scan_temp_bytes(E), 256);
}

sssp_status compact_launch(const sssp_graph* g, const uint8_t* keep, uint32_t* row_ptr_out, uint32_t* col_out,
                           uint32_t* w_out, uint32_t* emap_out, uint32_t* E_out, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    if (ws_bytes < compact_workspace_bytes(g->V, g->E)) return SSSP_ENOMEM;
    char* p = static_cast<char*>(ws);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(p);
    uint32_t* flags = reinterpret_cast<uint32_t*>(p + WS_HEADER_BYTES);
    uint32_t* pos = reinterpret_cast<uint32_t*>(p + WS_HEADER_BYTES + align_up(4ull * std::max<uint32_t>(g->E, 1), 256));
    void* tmp = p + WS_HEADER_BYTES + 2 * align_up(4ull * std::max<uint32_t>(g->E, 1), 256);
    CK(cudaMemsetAsync(hdr, 0, WS_HEADER_BYTES, st));
    const unsigned gr = grid_for(std::max<uint64_t>(g->E, (uint64_t)g->V + 1));
    if (g->E) {
        k_keep_u32<<<gr, 256, 0, st>>>(g->E, keep, flags);
        CK(cudaGetLastError());
        CK(inclusive_scan_u32(tmp, flags, pos, g->E, st));
    }
    k_compact<<<gr, 256, 0, st>>>(g->V, g->E, g->row_ptr, g->col, static_cast<const uint32_t*>(g->w), keep, pos,
                                  row_ptr_out, col_out, w_out, emap_out, E_out);
    CK(cudaGetLastError());
    return SSSP_OK;
}

}  // namespace sssp
