// The Trishla test of Sec. III.B (Algorithm 1) on one chunk of consecutive edges, by one warp.
// Shared by the stand-alone prune kernel (prune.cu) and by idle blocks of the persistent
// solve (relax.cu), which prune while they wait for messages (the paper's use of idle time).
//
// The lanes read 32 edges (u, v_i) of the chunk at a time (their tails found inside the
// chunk's row range) and a ballot picks the ones whose v_i may serve as a witness (local mode:
// v_i in u's partition); for each of those the whole warp intersects the sorted adjacency
// lists N(u) and N(v_i) -- walking the shorter and binary-searching the longer -- and for
// every common head v_j tests  w(u, v_j) > w(u, v_i) + w(v_i, v_j).  A hit clears
// keep[(u, v_j)] and lowers witness[(u, v_j)] to v_i with atomicMin, so the recorded witness
// is the smallest one whatever the schedule.  All reads are of the unpruned graph (a
// snapshot), so the result does not depend on the order in which chunks run.
#pragma once

#include "common.cuh"

namespace sssp {

__device__ __forceinline__ uint32_t tri_lower_bound(const uint32_t* a, uint32_t lo, uint32_t hi, uint32_t x) {
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
__device__ __forceinline__ bool tri_dominated(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj);

template <>
__device__ __forceinline__ bool tri_dominated<WU32>(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj) {
    return (unsigned long long)w_uvj > (unsigned long long)w_uvi + w_vivj;
}

template <>
__device__ __forceinline__ bool tri_dominated<WF32>(uint32_t w_uvj, uint32_t w_uvi, uint32_t w_vivj) {
    return __uint_as_float(w_uvj) > __fadd_rn(__uint_as_float(w_uvi), __uint_as_float(w_vivj));
}

// the row (tail) of edge e: the largest r in [lo, hi) with row_ptr[r] <= e (row_ptr[lo] <= e)
__device__ __forceinline__ uint32_t tri_row_of(const uint32_t* row_ptr, uint32_t lo, uint32_t hi, uint32_t e) {
    while (hi - lo > 1u) {
        const uint32_t m = (lo + hi) >> 1;
        if (__ldg(&row_ptr[m]) <= e)
            lo = m;
        else
            hi = m;
    }
    return lo;
}

// Where a Trishla job stands: the graph, the chunking and the outputs.
struct TrishlaJob {
    uint32_t V, E, chunk, nchunks;
    unsigned long long B;  // partition block size (local mode)
    int mode;              // 0 local, 1 global
    const uint32_t* row_ptr;
    const uint32_t* col;
    const uint32_t* w;
    uint8_t* keep;
    uint32_t* witness;  // may be NULL
};

// Which candidate pairs (u, v_i) a call tests: all, only the light ones (both adjacency lists
// at most TRISHLA_LIGHT long: a few dependent loads, so a solve block that runs them between
// its rounds stays responsive), or only the heavy ones (the rest).  Tests are idempotent, so a
// pair may be tested once or twice; splitting a chunk's pairs into light and heavy covers each.
enum : int { TRI_ALL = 0, TRI_LIGHT = 1, TRI_HEAVY = 2 };
constexpr uint32_t TRISHLA_LIGHT = 64;

// Chunk `ch` (< J.nchunks) of the job, by the calling warp (all 32 lanes).
template <class W>
__device__ __noinline__ void trishla_chunk(const TrishlaJob& J, uint32_t ch, int which = TRI_ALL) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t e0 = ch * J.chunk, e1 = min(e0 + J.chunk, J.E);
    const uint32_t r0 = tri_row_of(J.row_ptr, 0u, J.V, e0);
    const uint32_t r1 = tri_row_of(J.row_ptr, r0, J.V, e1 - 1u) + 1u;  // rows of the chunk: [r0, r1)
    for (uint32_t base = e0; base < e1; base += 32u) {
        const uint32_t ei = base + lane;
        const bool in = ei < e1;
        const uint32_t u = in ? tri_row_of(J.row_ptr, r0, r1, ei) : r0;
        const uint32_t vi = in ? __ldg(&J.col[ei]) : NONE;
        const bool cand = vi < J.V && (J.mode != 0 || (unsigned long long)vi / J.B == (unsigned long long)u / J.B);
        uint32_t ball = __ballot_sync(0xFFFFFFFFu, cand);
        while (ball) {
            const uint32_t f = __ffs(ball) - 1u;
            ball &= ball - 1u;
            const uint32_t uu = __shfl_sync(0xFFFFFFFFu, u, f);
            const uint32_t v = __shfl_sync(0xFFFFFFFFu, vi, f);
            const uint32_t w_uvi = __ldg(&J.w[base + f]);
            const uint32_t a0 = __ldg(&J.row_ptr[uu]), a1 = __ldg(&J.row_ptr[uu + 1]);
            const uint32_t b0 = __ldg(&J.row_ptr[v]), b1 = __ldg(&J.row_ptr[v + 1]);
            if (which != TRI_ALL && ((max(a1 - a0, b1 - b0) <= TRISHLA_LIGHT) != (which == TRI_LIGHT))) continue;
            if (a1 - a0 <= b1 - b0) {
                // walk N(u), search N(v_i)
                for (uint32_t j = a0 + lane; j < a1; j += 32u) {
                    const uint32_t vj = __ldg(&J.col[j]);
                    const uint32_t k = tri_lower_bound(J.col, b0, b1, vj);
                    if (k < b1 && __ldg(&J.col[k]) == vj && tri_dominated<W>(__ldg(&J.w[j]), w_uvi, __ldg(&J.w[k]))) {
                        J.keep[j] = 0;
                        if (J.witness) atomicMin(&J.witness[j], v);
                    }
                }
            } else {
                // walk N(v_i), search N(u)
                for (uint32_t k = b0 + lane; k < b1; k += 32u) {
                    const uint32_t vj = __ldg(&J.col[k]);
                    const uint32_t j = tri_lower_bound(J.col, a0, a1, vj);
                    if (j < a1 && __ldg(&J.col[j]) == vj && tri_dominated<W>(__ldg(&J.w[j]), w_uvi, __ldg(&J.w[k]))) {
                        J.keep[j] = 0;
                        if (J.witness) atomicMin(&J.witness[j], v);
                    }
                }
            }
        }
    }
}

}  // namespace sssp
