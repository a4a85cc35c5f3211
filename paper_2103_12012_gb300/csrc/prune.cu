// K3 Trishla triangle prune (Sec. III.B, Algorithm 1).
//
// One warp per chunk of consecutive edges, 32 edges (u, v_i) at a time: for
// each one whose v_i may be a witness, the warp intersects the sorted adjacency
// lists N(u) and N(v_i) -- lanes walk the shorter list and binary-search each
// entry in the longer one -- and for every common head v_j tests
//     w(u, v_j) > w(u, v_i) + w(v_i, v_j).
// A hit clears keep[(u, v_j)] and lowers witness[(u, v_j)] to v_i with
// atomicMin, so the recorded witness is the smallest one whatever the
// schedule.  In local mode (the paper's "(v_i, v_j) in E_i") the pair is only
// considered when v_i lies in u's partition.  All reads are of the unpruned
// graph, so the result is the same as evaluating Algorithm 1 on a snapshot.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sssp {
namespace {

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t x) {
    while (lo < hi) {
        const uint32_t m = lo + ((hi - lo) >> 1);
        if (__ldg(&a[m]) < x)
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

template <class W>
__device__ __forceinline__ bool dominated(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj);

template <>
__device__ __forceinline__ bool dominated<WU32>(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj) {
    return (unsigned long long)w_uvj > (unsigned long long)w_uvi + w_vivj;
}

template <>
__device__ __forceinline__ bool dominated<WF32>(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj) {
    return __uint_as_float(w_uvj) > __fadd_rn(__uint_as_float(w_uvi), __uint_as_float(w_vivj));
}

constexpr uint32_t TRISHLA_CHUNK_MAX = 1024;  // consecutive edges one warp takes at most (hub rows spread over warps)

// the row (tail) of edge e: the largest r in [lo, hi) with row_ptr[r] <= e (row_ptr[lo] <= e)
__device__ __forceinline__ uint32_t row_of(const uint32_t* row_ptr, uint32_t lo, uint32_t hi, uint32_t e) {
    while (hi - lo > 1u) {
        const uint32_t m = (lo + hi) >> 1;
        if (__ldg(&row_ptr[m]) <= e)
            lo = m;
        else
            hi = m;
    }
    return lo;
}

template <class W>
__global__ void __launch_bounds__(256) k_trishla(uint32_t V, uint32_t E, uint32_t chunk, unsigned long long B, int mode,
                                                 const uint32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
                                                 const uint32_t* __restrict__ w, uint8_t* keep, uint32_t* witness) {
    // One warp per chunk of `chunk` consecutive edges: the lanes read 32 edges (u, v_i)
    // at a time (their tails found inside the chunk's row range) and a ballot picks the ones
    // whose v_i may serve as a witness (local mode: v_i in u's partition); for each of those
    // the whole warp intersects N(u) with N(v_i), walking the shorter list and binary-searching
    // the longer.
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t nchunks = (E + chunk - 1u) / chunk;
    for (uint32_t ch = warp; ch < nchunks; ch += nwarps) {
        const uint32_t e0 = ch * chunk, e1 = min(e0 + chunk, E);
        const uint32_t r0 = row_of(row_ptr, 0u, V, e0);
        const uint32_t r1 = row_of(row_ptr, r0, V, e1 - 1u) + 1u;  // rows of the chunk: [r0, r1)
        for (uint32_t base = e0; base < e1; base += 32u) {
            const uint32_t ei = base + lane;
            const bool in = ei < e1;
            const uint32_t u = in ? row_of(row_ptr, r0, r1, ei) : r0;
            const uint32_t vi = in ? __ldg(&col[ei]) : NONE;
            const bool cand = vi < V && (mode != 0 || (unsigned long long)vi / B == (unsigned long long)u / B);
            uint32_t ball = __ballot_sync(0xFFFFFFFFu, cand);
            while (ball) {
                const uint32_t f = __ffs(ball) - 1u;
                ball &= ball - 1u;
                const uint32_t uu = __shfl_sync(0xFFFFFFFFu, u, f);
                const uint32_t v = __shfl_sync(0xFFFFFFFFu, vi, f);
                const uint32_t w_uvi = __ldg(&w[base + f]);
                const uint32_t a0 = __ldg(&row_ptr[uu]), a1 = __ldg(&row_ptr[uu + 1]);
                const uint32_t b0 = __ldg(&row_ptr[v]), b1 = __ldg(&row_ptr[v + 1]);
                if (a1 - a0 <= b1 - b0) {
                    // walk N(u), search N(v_i)
                    for (uint32_t j = a0 + lane; j < a1; j += 32u) {
                        const uint32_t vj = __ldg(&col[j]);
                        const uint32_t k = lower_bound_u32(col, b0, b1, vj);
                        if (k < b1 && __ldg(&col[k]) == vj && dominated<W>(__ldg(&w[j]), w_uvi, __ldg(&w[k]))) {
                            keep[j] = 0;
                            if (witness) atomicMin(&witness[j], v);
                        }
                    }
                } else {
                    // walk N(v_i), search N(u)
                    for (uint32_t k = b0 + lane; k < b1; k += 32u) {
                        const uint32_t vj = __ldg(&col[k]);
                        const uint32_t j = lower_bound_u32(col, a0, a1, vj);
                        if (j < a1 && __ldg(&col[j]) == vj && dominated<W>(__ldg(&w[j]), w_uvi, __ldg(&w[k]))) {
                            keep[j] = 0;
                            if (witness) atomicMin(&witness[j], v);
                        }
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t prune_launch(const sssp_graph* g, int mode, uint8_t* keep, uint32_t* witness, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(keep, 1, g->E, st)) != cudaSuccess) return e;
    if (witness && (e = cudaMemsetAsync(witness, 0xFF, sizeof(uint32_t) * (size_t)g->E, st)) != cudaSuccess) return e;
    if (g->E == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned long long B = ((unsigned long long)g->V + g->partitions - 1) / g->partitions;
    // chunks: enough for about 128 warps per SM, between 32 and TRISHLA_CHUNK_MAX edges each
    uint32_t chunk = 32;
    while (chunk < TRISHLA_CHUNK_MAX && (uint64_t)g->E / (2ull * chunk) >= (uint64_t)sms * 128) chunk *= 2;
    const uint64_t want = (((uint64_t)g->E + chunk - 1) / chunk * 32 + 255) / 256;  // a warp per chunk
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 32));
    const uint32_t* w = static_cast<const uint32_t*>(g->w);
    if (g->wtype == SSSP_W_F32)
        k_trishla<WF32><<<grid, 256, 0, st>>>(g->V, g->E, chunk, B, mode, g->row_ptr, g->col, w, keep, witness);
    else
        k_trishla<WU32><<<grid, 256, 0, st>>>(g->V, g->E, chunk, B, mode, g->row_ptr, g->col, w, keep, witness);
    return cudaGetLastError();
}

}  // namespace sssp
