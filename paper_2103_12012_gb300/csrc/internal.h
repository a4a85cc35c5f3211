// Host-side interfaces between the C-ABI layer (api.cu) and the kernel files.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "sssp.h"
#include "trishla.cuh"

namespace sssp {

struct WsHeader;

// ------------------------------------------------------------------ relax.cu
struct SolveLaunch {
    // graph
    const uint32_t* row_ptr;
    const uint32_t* col;
    const uint32_t* w;
    int wtype;
    uint32_t V;
    const uint32_t* ids;    // stored vertex -> caller's id (NULL: identity)
    const uint32_t* slots;  // caller's id -> stored vertex (NULL: identity)
    // problems
    uint32_t S;
    const uint32_t* sources;
    // ownership
    uint32_t B;      // partition block size ceil(V/P)
    uint32_t Bq;     // sub-block size ceil(B/split)
    uint32_t split;  // sub-blocks per partition
    uint32_t Q;      // units per source = P*split
    uint32_t words;  // bitmap words per source
    // workspace views
    WsHeader* hdr;
    unsigned long long* packed;  // [S][V]
    uint32_t* bitmap;            // [S][words]
    uint32_t* dirty;             // [S*Q]
    uint32_t* nfsplit;           // [S*Q] near-far split point per unit
    // schedule
    uint32_t threads, tile, grid;
    uint32_t delta_bits;
    uint32_t policy;      // SSSP_POLICY_*
    uint32_t msg_buffer;  // 0: direct messages, else the push-out size
    uint32_t hub_count;   // layout graphs: the first hub_count stored vertices of each partition are hubs
    uint32_t hub_delta_bits;  // bucket width of hubs (a quarter of delta)
    uint32_t hub_mid_bits;    // bucket width of the next 3 * hub_count vertices (half of delta)
    uint64_t timeout_ns;
    uint32_t hold_pending;
    cudaEvent_t ev_begin, ev_end;  // optional timing events around the relaxation kernel
    // outputs (and, for a warm start, the previous result they start from)
    uint32_t* dist;
    uint32_t* pred;
    // warm start: tails of the edges whose weight fell or that were added
    uint32_t warm;
    const uint32_t* warm_tails;
    uint32_t n_tails;
    // prune while idle (sssp_solve_prune): blocks with no dirty unit run Trishla chunks
    uint32_t prune_on;
    TrishlaJob prune;
};

constexpr uint32_t SOLVE_MAX_THREADS = 512;   // block size limit of the solve kernel
constexpr uint32_t BATCH_MAX_THREADS = 1024;  // block size limit of the batched kernel
size_t relax_smem_bytes(uint32_t tile, uint32_t Q, bool msgs);
cudaError_t relax_max_blocks_per_sm(int wtype, uint32_t threads, uint32_t tile, uint32_t Q, int* out,
                                    bool prune = false, bool msgs = false, bool hubs = false);
cudaError_t launch_solve(const SolveLaunch& L, cudaStream_t st);

// One problem of a batch, in the order blocks take them (largest first).
struct BatchProblem {
    unsigned long long row_off, edge_off, out_off, bm_off;
    uint32_t V, src, E, pad;
};
static_assert(sizeof(BatchProblem) == 48, "batch problem layout");

struct BatchLaunch {
    const uint32_t* row_ptr;
    const uint32_t* col;
    const uint32_t* w;
    int wtype;
    uint32_t n_problems;
    const BatchProblem* probs;  // device
    WsHeader* hdr;
    unsigned long long* packed;  // [sum V]
    uint32_t* bitmap;
    uint32_t threads, tile, grid;
    uint32_t delta_bits;
    uint64_t timeout_ns;
    uint32_t* dist;
    uint32_t* pred;
    cudaEvent_t ev_begin, ev_end;
};

uint32_t batched_bitmaps();  // inbox bitmaps per batched problem (distance buckets + overflow)
cudaError_t batched_max_blocks_per_sm(int wtype, uint32_t threads, uint32_t tile, int* out);
cudaError_t launch_batched(const BatchLaunch& L, cudaStream_t st);

// -------------------------------------------------------------------- csr.cu
size_t csr_workspace_bytes(uint32_t V, uint64_t E_raw);
sssp_status csr_build(uint32_t V, uint64_t E_raw, const uint32_t* src, const uint32_t* dst, const uint32_t* w,
                      int wtype, uint32_t* row_ptr, uint32_t* col, uint32_t* w_out, uint32_t* eid, uint32_t* E_out,
                      void* ws, size_t ws_bytes, cudaStream_t st);
cudaError_t partition_launch(const sssp_graph* g, uint32_t* bounds, uint64_t* inter, cudaStream_t st);
size_t layout_workspace_bytes(uint32_t V, uint32_t E);
sssp_status layout_build(const sssp_graph* g, uint32_t* row_ptr_out, uint32_t* col_out, uint32_t* w_out,
                         uint32_t* emap_out, uint32_t* ids_out, uint32_t* slots_out, void* ws, size_t ws_bytes,
                         cudaStream_t st);
size_t compact_workspace_bytes(uint32_t V, uint32_t E);
sssp_status compact_launch(const sssp_graph* g, const uint8_t* keep, uint32_t* row_ptr_out, uint32_t* col_out,
                           uint32_t* w_out, uint32_t* emap_out, uint32_t* E_out, void* ws, size_t ws_bytes,
                           cudaStream_t st);

// ------------------------------------------------------------------- sort.cu
// stable LSD radix sort of (key, value) pairs on key bits [0, end_bit), ping-ponging between
// (k0, v0) and (k1, v1); *in_second tells which pair of buffers holds the result
size_t sort_temp_bytes(uint64_t n);
cudaError_t sort_pairs_u64(void* tmp, unsigned long long* k0, unsigned long long* k1, uint32_t* v0, uint32_t* v1,
                           uint64_t n, int end_bit, cudaStream_t st, bool* in_second);
size_t scan_temp_bytes(uint64_t n);
cudaError_t inclusive_scan_u32(void* tmp, const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t st);

// ------------------------------------------------------------------ prune.cu
cudaError_t prune_launch(const sssp_graph* g, int mode, uint8_t* keep, uint32_t* witness, cudaStream_t st);
TrishlaJob trishla_job(const sssp_graph* g, int mode, uint8_t* keep, uint32_t* witness);
cudaError_t trishla_init(const TrishlaJob& J, cudaStream_t st);  // keep = 1, witness = NONE
// every pair of every chunk (cursor NULL), or what a solve's idle blocks left of the job: the
// heavy pairs of the chunks below *cursor and every pair of the others
cudaError_t trishla_launch(const TrishlaJob& J, int wtype, const unsigned long long* cursor, cudaStream_t st);

// --------------------------------------------------------------- backward.cu
size_t backward_workspace_bytes(uint32_t V, uint32_t E, uint32_t S);
cudaError_t backward_launch(const sssp_graph* g, uint32_t S, const uint32_t* pred, const float* grad_dist,
                            float* grad_w, void* ws, cudaStream_t st);

// ------------------------------------------------------------------- common
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
constexpr size_t WS_HEADER_BYTES = 256;

}  // namespace sssp
