// K3 Trishla triangle prune (Sec. III.B, Algorithm 1).
//
// One warp per chunk of consecutive edges (trishla.cuh): for each edge (u, v_i) whose v_i may
// be a witness, the warp intersects the sorted adjacency lists N(u) and N(v_i) and clears
// keep[(u, v_j)] where w(u, v_j) > w(u, v_i) + w(v_i, v_j), recording the least witness.  In
// local mode (the paper's "(v_i, v_j) in E_i") only v_i in u's partition is considered.  The
// stand-alone launch tests every pair of every chunk; the launch that finishes a job begun by the
// idle blocks of a solve (sssp_solve_prune) tests the heavy pairs of the chunks they took and
// every pair of the rest.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "trishla.cuh"

namespace sssp {
namespace {

// Consecutive edges one warp takes.  Small chunks spread the rows of hub vertices (whose pairs
// cost the most) over many warps: on R-MAT scale 22 (148 partitions, local mode) 32-edge chunks
// take 8.8 ms against 17.9 ms for chunks grown to 1,024 edges; on a triangle-free grid they cost
// 9.2 against 7.9 ms.
constexpr uint32_t TRISHLA_CHUNK = 32;

// Warp w takes chunks w, w + nwarps, ...  With a cursor (the end of a job the idle blocks of a
// solve began: they handed out chunks [0, *cursor) and tested their light pairs) the chunks
// below the cursor get their heavy pairs only, the others every pair.
template <class W>
__global__ void __launch_bounds__(256) k_trishla(TrishlaJob J, const unsigned long long* cursor) {
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned long long done = cursor ? min(*cursor, (unsigned long long)J.nchunks) : 0ull;
    for (uint32_t ch = warp; ch < J.nchunks; ch += nwarps) trishla_chunk<W>(J, ch, ch < done ? TRI_HEAVY : TRI_ALL);
}

unsigned trishla_grid(const TrishlaJob& J) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = ((uint64_t)J.nchunks * 32 + 255) / 256;  // a warp per chunk
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 32));
}

}  // namespace

TrishlaJob trishla_job(const sssp_graph* g, int mode, uint8_t* keep, uint32_t* witness) {
    TrishlaJob J{};
    J.V = g->V;
    J.E = g->E;
    J.B = ((unsigned long long)g->V + g->partitions - 1) / g->partitions;
    J.mode = mode;
    J.row_ptr = g->row_ptr;
    J.col = g->col;
    J.w = static_cast<const uint32_t*>(g->w);
    J.keep = keep;
    J.witness = witness;
    J.chunk = TRISHLA_CHUNK;
    J.nchunks = (uint32_t)(((uint64_t)g->E + TRISHLA_CHUNK - 1) / TRISHLA_CHUNK);
    return J;
}

cudaError_t trishla_init(const TrishlaJob& J, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(J.keep, 1, J.E, st)) != cudaSuccess) return e;
    if (J.witness && (e = cudaMemsetAsync(J.witness, 0xFF, sizeof(uint32_t) * (size_t)J.E, st)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

cudaError_t trishla_launch(const TrishlaJob& J, int wtype, const unsigned long long* cursor, cudaStream_t st) {
    if (J.nchunks == 0) return cudaSuccess;
    const unsigned grid = trishla_grid(J);
    if (wtype == SSSP_W_F32)
        k_trishla<WF32><<<grid, 256, 0, st>>>(J, cursor);
    else
        k_trishla<WU32><<<grid, 256, 0, st>>>(J, cursor);
    return cudaGetLastError();
}

cudaError_t prune_launch(const sssp_graph* g, int mode, uint8_t* keep, uint32_t* witness, cudaStream_t st) {
    const TrishlaJob J = trishla_job(g, mode, keep, witness);
    cudaError_t e;
    if ((e = trishla_init(J, st)) != cudaSuccess) return e;
    return trishla_launch(J, g->wtype, nullptr, st);
}

}  // namespace sssp
