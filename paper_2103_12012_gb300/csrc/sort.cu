// Device-wide primitives of the one-time graph steps (CSR build, locality layout, compaction):
// a stable radix sort of (64-bit key, 32-bit value) pairs and a prefix sum of 32-bit counts.
//
// Sort: least-significant digit first, 8 bits a pass over the bits [0, end_bit) that the keys
// use.  A pass over n pairs cuts them into tiles of SORT_TILE (each thread holds SORT_ITEMS
// pairs in registers, a warp a contiguous run of 32 * SORT_ITEMS):
//   1. each tile counts its digits (shared atomics) into counts[digit * ntiles + tile];
//   2. an exclusive prefix sum of counts, digit-major, gives every (digit, tile) the first
//      output position of its pairs;
//   3. each tile orders its pairs by digit in shared memory: a warp ranks equal digits within
//      32 lanes with __match_any_sync and keeps a running count per digit, warps before it add
//      their digit counts, so pairs keep their input order within a digit (stable, which LSD
//      needs); the ordered tile then goes out run by run, consecutive threads storing
//      consecutive pairs of one digit.
// Scan: tiles of SCAN_TILE values staged in shared memory; a first kernel sums each tile, the
// tile sums are scanned (recursively while there are more than one tile of them), and a second
// kernel scans each tile from its offset.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sssp {
namespace {

constexpr uint32_t SORT_THREADS = 256;
constexpr uint32_t SORT_ITEMS = 8;                            // pairs a thread holds
constexpr uint32_t SORT_WARPS = SORT_THREADS / 32;
constexpr uint32_t SORT_WARP_RUN = 32 * SORT_ITEMS;           // consecutive pairs a warp takes
constexpr uint32_t SORT_TILE = SORT_THREADS * SORT_ITEMS;     // pairs a block takes
constexpr uint32_t RADIX = 256;

constexpr uint32_t SCAN_THREADS = 256;
constexpr uint32_t SCAN_ITEMS = 16;
constexpr uint32_t SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t digit_of(unsigned long long k, uint32_t shift) {
    return (uint32_t)(k >> shift) & (RADIX - 1u);
}

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ uint32_t block_excl(uint32_t x, uint32_t* wsum, uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31u) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (uint32_t o = 1; o < 32u; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    const uint32_t r = (warp ? wsum[warp - 1] : 0u) + inc - x;
    *total = wsum[nw - 1];
    __syncthreads();
    return r;
}

// 1. digit counts of each tile, digit-major
__global__ void __launch_bounds__(SORT_THREADS) k_sort_count(const unsigned long long* __restrict__ keys,
                                                             unsigned long long n, uint32_t shift, uint32_t ntiles,
                                                             uint32_t* counts) {
    __shared__ uint32_t hist[RADIX];
    const uint32_t tile = blockIdx.x;
    hist[threadIdx.x] = 0u;  // SORT_THREADS == RADIX
    __syncthreads();
    const unsigned long long base = (unsigned long long)tile * SORT_TILE;
    for (uint32_t i = threadIdx.x; i < SORT_TILE; i += SORT_THREADS) {
        const unsigned long long at = base + i;
        if (at < n) atomicAdd(&hist[digit_of(keys[at], shift)], 1u);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * ntiles + tile] = hist[threadIdx.x];
}

// 3. stable placement of each tile's pairs from the scanned counts: the tile is first ordered by
// digit in shared memory (stable), then written out so that consecutive threads store consecutive
// pairs of one digit's run (coalesced stores instead of a scatter)
__global__ void __launch_bounds__(SORT_THREADS) k_sort_place(const unsigned long long* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin, unsigned long long n,
                                                             uint32_t shift, uint32_t ntiles,
                                                             const uint32_t* __restrict__ offsets,
                                                             unsigned long long* kout, uint32_t* vout) {
    __shared__ uint32_t wcount[SORT_WARPS][RADIX];  // per warp: digit counts, then running positions
    __shared__ unsigned long long sk[SORT_TILE];
    __shared__ uint32_t sv[SORT_TILE];
    __shared__ uint32_t tstart[RADIX];  // first position of each digit in the tile's digit order
    __shared__ uint32_t gbase[RADIX];   // first output position of the tile's pairs of each digit
    __shared__ uint32_t wsum[32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, tile = blockIdx.x;
    for (uint32_t i = threadIdx.x; i < SORT_WARPS * RADIX; i += SORT_THREADS) (&wcount[0][0])[i] = 0u;
    __syncthreads();
    const unsigned long long tbase = (unsigned long long)tile * SORT_TILE;
    const unsigned long long wbase = tbase + (unsigned long long)warp * SORT_WARP_RUN;
    const uint32_t tcount = (uint32_t)min((unsigned long long)SORT_TILE, n - tbase);
    unsigned long long k[SORT_ITEMS];
    uint32_t v[SORT_ITEMS], d[SORT_ITEMS];
#pragma unroll
    for (uint32_t j = 0; j < SORT_ITEMS; ++j) {
        const unsigned long long at = wbase + j * 32u + lane;
        const bool in = at < n;
        k[j] = in ? kin[at] : 0ull;
        v[j] = in ? vin[at] : 0u;
        d[j] = in ? digit_of(k[j], shift) : RADIX;  // RADIX: no pair
    }
    // this warp's digit counts (one leader per digit group per step: no other writer)
#pragma unroll
    for (uint32_t j = 0; j < SORT_ITEMS; ++j) {
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d[j]);
        if (d[j] < RADIX && lane == (uint32_t)(__ffs(peers) - 1)) wcount[warp][d[j]] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // digit totals of the tile, their start in digit order, and each warp's running position
    {
        const uint32_t dg = threadIdx.x;  // SORT_THREADS == RADIX
        uint32_t tot = 0;
        for (uint32_t w = 0; w < SORT_WARPS; ++w) tot += wcount[w][dg];
        uint32_t all;
        const uint32_t start = block_excl(tot, wsum, &all);
        tstart[dg] = start;
        gbase[dg] = offsets[(size_t)dg * ntiles + tile];
        uint32_t run = start;
        for (uint32_t w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = wcount[w][dg];
            wcount[w][dg] = run;
            run += c;
        }
    }
    __syncthreads();
    // the tile in digit order (stable) in shared memory
#pragma unroll
    for (uint32_t j = 0; j < SORT_ITEMS; ++j) {
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d[j]);
        if (d[j] < RADIX) {
            const uint32_t pos = wcount[warp][d[j]] + (uint32_t)__popc(peers & ((1u << lane) - 1u));
            sk[pos] = k[j];
            sv[pos] = v[j];
        }
        __syncwarp();
        if (d[j] < RADIX && lane == (uint32_t)(__ffs(peers) - 1)) wcount[warp][d[j]] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < tcount; i += SORT_THREADS) {
        const unsigned long long key = sk[i];
        const uint32_t dg = digit_of(key, shift);
        const uint32_t pos = gbase[dg] + (i - tstart[dg]);
        kout[pos] = key;
        vout[pos] = sv[i];
    }
}

// --- scan

// sum of each tile
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(const uint32_t* __restrict__ in, unsigned long long n,
                                                            uint32_t* sums) {
    __shared__ uint32_t wsum[32];
    const unsigned long long base = (unsigned long long)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (uint32_t i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const unsigned long long at = base + i;
        if (at < n) s += in[at];
    }
    uint32_t total;
    block_excl(s, wsum, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// scan of each tile from its offset (offsets NULL: 0); inclusive or exclusive
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const uint32_t* __restrict__ in, unsigned long long n,
                                                             const uint32_t* __restrict__ offsets, uint32_t* out,
                                                             int inclusive) {
    __shared__ uint32_t tilev[SCAN_TILE];
    __shared__ uint32_t wsum[32];
    const unsigned long long base = (unsigned long long)blockIdx.x * SCAN_TILE;
    for (uint32_t i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const unsigned long long at = base + i;
        tilev[i] = at < n ? in[at] : 0u;
    }
    __syncthreads();
    uint32_t vals[SCAN_ITEMS], s = 0;
#pragma unroll
    for (uint32_t j = 0; j < SCAN_ITEMS; ++j) {
        vals[j] = tilev[threadIdx.x * SCAN_ITEMS + j];
        s += vals[j];
    }
    uint32_t total;
    uint32_t run = block_excl(s, wsum, &total) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
    for (uint32_t j = 0; j < SCAN_ITEMS; ++j) {
        tilev[threadIdx.x * SCAN_ITEMS + j] = inclusive ? run + vals[j] : run;
        run += vals[j];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        const unsigned long long at = base + i;
        if (at < n) out[at] = tilev[i];
    }
}

uint64_t tiles_of(uint64_t n, uint64_t tile) { return (n + tile - 1) / tile; }

// temp words the scan of n values needs: the tile sums of every level
size_t scan_temp_words(uint64_t n) {
    size_t w = 0;
    for (uint64_t m = tiles_of(n, SCAN_TILE); m > 1; m = tiles_of(m, SCAN_TILE)) w += align_up(m, 64);
    return w + 64;
}

cudaError_t scan_u32(uint32_t* tmp, const uint32_t* in, uint32_t* out, uint64_t n, bool inclusive, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint64_t nt = tiles_of(n, SCAN_TILE);
    if (nt == 1) {
        k_scan_tiles<<<1, SCAN_THREADS, 0, st>>>(in, n, nullptr, out, inclusive ? 1 : 0);
        return cudaGetLastError();
    }
    uint32_t* sums = tmp;
    uint32_t* rest = tmp + align_up(nt, 64);
    k_scan_sums<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = scan_u32(rest, sums, sums, nt, false, st)) != cudaSuccess) return e;  // tile offsets, in place
    k_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, st>>>(in, n, sums, out, inclusive ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

size_t sort_temp_bytes(uint64_t n) {
    const uint64_t ntiles = std::max<uint64_t>(tiles_of(n, SORT_TILE), 1);
    const uint64_t ncounts = RADIX * ntiles;
    return 4 * (align_up(ncounts, 64) + scan_temp_words(ncounts));
}

size_t scan_temp_bytes(uint64_t n) { return 4 * scan_temp_words(n); }

cudaError_t inclusive_scan_u32(void* tmp, const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t st) {
    return scan_u32(static_cast<uint32_t*>(tmp), in, out, n, true, st);
}

cudaError_t sort_pairs_u64(void* tmp, unsigned long long* k0, unsigned long long* k1, uint32_t* v0, uint32_t* v1,
                           uint64_t n, int end_bit, cudaStream_t st, bool* in_second) {
    *in_second = false;
    if (n <= 1 || end_bit <= 0) return cudaSuccess;
    const uint64_t ntiles = tiles_of(n, SORT_TILE);
    uint32_t* counts = static_cast<uint32_t*>(tmp);
    uint32_t* scan_tmp = counts + align_up(RADIX * ntiles, 64);
    cudaError_t e;
    for (int shift = 0; shift < end_bit; shift += 8) {
        k_sort_count<<<(unsigned)ntiles, SORT_THREADS, 0, st>>>(k0, n, (uint32_t)shift, (uint32_t)ntiles, counts);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = scan_u32(scan_tmp, counts, counts, RADIX * ntiles, false, st)) != cudaSuccess) return e;
        k_sort_place<<<(unsigned)ntiles, SORT_THREADS, 0, st>>>(k0, v0, n, (uint32_t)shift, (uint32_t)ntiles, counts,
                                                                k1, v1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::swap(k0, k1);
        std::swap(v0, v1);
        *in_second = !*in_second;
    }
    return cudaSuccess;
}

}  // namespace sssp
