/*
 * sssp.h -- C ABI of libsssp, a GB300 (sm_103a) implementation of the hot
 * path of SP_Async (S. Yadav, A. Khan, "SP_Async: Single Source Shortest Path
 * in Asynchronous Mode on MPI", arXiv 2103.12012).
 *
 * The paper's problem (Sec. I): a directed graph G(V,E) with non-negative
 * edge costs W and a source S; find the least-cost path from S to every
 * vertex.  Its method (Sec. III): 1D block partitioning (Sec. III.A), the
 * Trishla triangle edge prune (Sec. III.B, Algorithm 1), Dijkstra inside each
 * partition and asynchronous Bellman-Ford-style messages between partitions
 * (Sec. III.C, SP-Async and DIJKSTRA), stopped by message-count termination
 * detection (Sec. III.D, ToKa).  On one GPU each partition is owned by a
 * persistent thread block, a message is a 64-bit atomicMin on the packed word
 * (distance << 32 | predecessor) of the target vertex plus a bit in the owner
 * partition's device-memory inbox, and termination is a device-global count
 * of queued-but-unprocessed vertices.
 *
 * Conventions shared by every entry point:
 *  - Ownership: the caller allocates and owns every buffer, device or host;
 *    the library allocates no device memory.  Scratch space ("workspace") is
 *    sized by the matching *_workspace_size query and passed in.
 *  - Pointers marked "device" must be device memory of the current device;
 *    "host" pointers are host memory.  Device buffers need 16-byte alignment
 *    (torch allocations satisfy this).
 *  - Streams: every call is asynchronous on `stream` (a cudaStream_t, NULL =
 *    the legacy default stream) unless it says otherwise.  Host-detectable
 *    argument errors return SSSP_EINVAL (or SSSP_ENOMEM for a workspace that
 *    is too small) before anything is launched.  Errors found on the device
 *    (timeout, overflow, bad weight, bad vertex id) are recorded in the
 *    workspace's status word; sssp_workspace_status() synchronises the stream
 *    and returns them.
 *  - Graph format (sssp_graph): CSR with 32-bit offsets and vertex ids; rows
 *    sorted by head, no self-loops, no parallel edges (sssp_build_csr makes
 *    this form).  Weights are uint32 >= 1 or float32 > 0 and finite.
 *  - Values: an unreachable vertex has dist 0xFFFFFFFF (uint32) or +inf
 *    (float32) and pred 0xFFFFFFFF; the source has dist 0 and pred
 *    0xFFFFFFFF.  pred[v] is the smallest vertex id u with
 *    dist(u) + w(u,v) == dist(v) (the canonical predecessor).
 *  - uint32 distances: a candidate d(u)+w that does not fit below 0xFFFFFFFF
 *    is discarded and the status becomes SSSP_EOVERFLOW; vertices whose true
 *    distance does not fit are then reported unreachable.
 */
#ifndef SSSP_H
#define SSSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sssp_stream_t; /* identical to cudaStream_t */

typedef enum {
    SSSP_OK = 0,
    SSSP_EINVAL = 1,     /* bad argument (host check) or bad vertex id / weight (device check) */
    SSSP_ENOMEM = 2,     /* workspace smaller than the size query asked for */
    SSSP_ECUDA = 3,      /* a CUDA runtime call failed */
    SSSP_ETIMEOUT = 4,   /* a device wait exceeded its limit; outputs are not valid */
    SSSP_EOVERFLOW = 5,  /* a uint32 path length exceeded 0xFFFFFFFE (see conventions) */
    SSSP_EINTERNAL = 6,  /* an internal invariant failed */
    SSSP_EUNSUPPORTED = 7
} sssp_status;

typedef enum { SSSP_W_U32 = 0, SSSP_W_F32 = 1 } sssp_wtype;

/* A CSR graph in device memory (Sec. III.A: the per-process adjacency Padj,
 * here one array for all partitions; partition p owns the vertex block
 * [p*B, min((p+1)*B, V)) with B = ceil(V / partitions)). */
typedef struct {
    uint32_t V;              /* vertex count, >= 1 */
    uint32_t E;              /* edge count */
    const uint32_t* row_ptr; /* device [V+1], row_ptr[0] = 0, row_ptr[V] = E */
    const uint32_t* col;     /* device [E], heads, strictly increasing within a row, != tail */
    const void* w;           /* device [E], uint32 or float32 according to wtype */
    int32_t wtype;           /* sssp_wtype */
    uint32_t partitions;     /* P >= 1 (Sec. III.A 1D block partitioning) */
    /* A graph from sssp_layout (both set) or a graph in the caller's own ids (both NULL).
     * For sssp_solve / sssp_autotune / sssp_solve_noalloc on a layout graph, sources
     * are given, and dist / pred are written, in the caller's ids, with the same values
     * (canonical predecessors included) as on the original graph.  sssp_partition,
     * sssp_prune and sssp_compact work on the CSR as stored; sssp_backward rejects a
     * layout graph (SSSP_EINVAL). */
    const uint32_t* ids;     /* device [V] or NULL: caller's id of stored vertex v */
    const uint32_t* slots;   /* device [V] or NULL: stored vertex of caller's id i (inverse of ids) */
} sssp_graph;

/* Tuning knobs; a zero field means "default".  None of them changes the
 * result, only the schedule. */
typedef struct {
    uint32_t threads;      /* threads per block of the relaxation kernel: a multiple of 32, 128..512 for
                              sssp_solve, 128..1024 for sssp_solve_batched (default 512) */
    uint32_t blocks_per_sm;/* persistent blocks per SM (default: as many as fit) */
    uint32_t tile;         /* most vertices one block takes from its inbox per round: 32..4096 (default 1024) */
    uint32_t split;        /* blocks sharing one partition, each owning a sub-block of its vertices (default 1) */
    double delta;          /* bucket width: a round takes inbox vertices with dist < min dist + delta
                              (default: uint32 -> 4, float32 -> 0.0625) */
    uint64_t timeout_ns;   /* limit on a block's continuous idle wait (default 20 s); a persistent
                              kernel also stops after 3 x timeout_ns in total */
    uint32_t flags;        /* SSSP_FLAG_* */
    uint32_t policy;       /* sssp_policy: which queued vertices a round of sssp_solve takes (default
                              SSSP_POLICY_RELATIVE); sssp_solve_batched keeps its own fixed buckets */
    uint32_t msg_buffer;   /* message buffering in sssp_solve (the push-out criteria Sec. VI leaves as
                              future work): 0 = direct, every message (an improvement of a vertex
                              owned by another unit) made visible to its owner at once; k in 1..32 =
                              a warp holds its messages and pushes them out, with one release fence,
                              once it holds k of them (size criterion) and at the end of every
                              sub-round (age criterion).  Messages inside a unit are never held. */
    uint32_t hub_count;    /* on a graph from sssp_layout (vertices stored by degree, highest first, inside
                              each partition): the first hub_count stored vertices of every partition
                              are hubs, which a round of sssp_solve takes only while their distance is
                              within delta / 4 of the unit's minimum, and the next 3 * hub_count
                              within delta / 2 (0 = no hubs; ignored on other graphs).  Processing a
                              high-degree vertex twice costs its whole row, so these wait for a
                              narrower bucket while the other vertices may take a wider one. */
    void* ev_relax_begin;  /* cudaEvent_t or NULL: recorded on `stream` right before the relaxation kernel */
    void* ev_relax_end;    /* cudaEvent_t or NULL: recorded right after it (for timing that kernel alone) */
} sssp_options;

/* Frontier policies of sssp_solve: how a round picks, among its unit's queued
 * vertices, the bucket it relaxes -- the approximation of Dijkstra's pop order
 * inside a partition (Sec. III.C, DIJKSTRA) that trades asynchrony against
 * wasted relaxations, as the Delta-stepping of the related work (Sec. II) does.
 * All give the same distances and predecessors; dmin is the least distance
 * queued in the unit when the round starts.
 *   RELATIVE : dist < dmin + delta
 *   FIXED    : dist < the end of the fixed bucket [k*delta, (k+1)*delta) holding dmin
 *   NEAR_FAR : dist < the unit's split point, which moves to dmin + delta whenever
 *              no queued vertex lies below it (near-far worklists: late messages
 *              below the split join the current near set instead of narrowing it)
 *   ALL      : every queued vertex (asynchronous Bellman-Ford; delta unused) */
typedef enum {
    SSSP_POLICY_RELATIVE = 0,
    SSSP_POLICY_FIXED = 1,
    SSSP_POLICY_NEAR_FAR = 2,
    SSSP_POLICY_ALL = 3
} sssp_policy;

/* Test hook: start the pending count one above the true value so that the
 * termination count can never reach zero; the solve must then end with
 * SSSP_ETIMEOUT after `timeout_ns`, with the device still usable. */
#define SSSP_FLAG_TEST_HOLD_PENDING 0x1u

/* Device-side counters of the last solve (sssp_workspace_status). */
typedef struct {
    uint64_t edges_scanned;    /* relaxations attempted: edges of every processed vertex */
    uint64_t atomics;          /* 64-bit atomicMin issued after the read-first filter */
    uint64_t improved;         /* atomicMin that lowered the target's distance */
    uint64_t activations;      /* inbox bits turned on (vertices queued) */
    uint64_t rounds;           /* rounds run by all blocks */
    uint64_t vertices;         /* vertices processed (taken from an inbox) */
    uint64_t remote_activations; /* activations of a vertex owned by another unit (messages, Alg. 3 send_msg) */
    uint64_t idle_us;          /* microseconds blocks spent waiting with no unit to process, summed over blocks */
    uint64_t prune_chunks;     /* sssp_solve_prune: Trishla chunks run by idle blocks during the solve */
} sssp_stats;

const char* sssp_status_string(sssp_status s);

/* Library build identity (a constant string). */
const char* sssp_version(void);

/* ------------------------------------------------------------------ K1 CSR */

/* Workspace bytes needed by sssp_build_csr for V vertices and E_raw input edges. */
size_t sssp_build_csr_workspace_size(uint32_t V, uint64_t E_raw);

/*
 * COO -> canonical CSR (the Padj adjacency of Sec. III.A).  Self-loops are
 * dropped and parallel edges collapsed to their minimum weight (lowest input
 * index on ties); neither changes any shortest distance.
 *   src, dst : device [E_raw] uint32 tail/head ids (< V, else SSSP_EINVAL on the device status)
 *   w        : device [E_raw] weights of type wtype
 *   row_ptr  : device [V+1] out
 *   col, w_out, eid : device [E_raw] out (first *E_out entries valid); eid[e] = input index of kept edge e
 *                     (eid may be NULL)
 *   E_out    : device [1] out, number of CSR edges
 *   ws       : device workspace of ws_bytes >= sssp_build_csr_workspace_size(V, E_raw); it also
 *              holds the status word read by sssp_workspace_status
 * E_raw must be < 2^32.
 */
sssp_status sssp_build_csr(uint32_t V, uint64_t E_raw, const uint32_t* src, const uint32_t* dst, const void* w,
                           int32_t wtype, uint32_t* row_ptr, uint32_t* col, void* w_out, uint32_t* eid,
                           uint32_t* E_out, void* ws, size_t ws_bytes, sssp_stream_t stream);

/* ------------------------------------------------------- K1b locality layout */

/* Workspace bytes of sssp_layout for graph g (0 if g is invalid or already a layout graph). */
size_t sssp_layout_workspace_size(const sssp_graph* g);

/*
 * The same graph with its vertices renumbered inside each 1D block partition
 * (Sec. III.A: partition membership, hence every partition's vertex count and
 * inter-edges, is unchanged): within a partition, by total degree (in + out)
 * descending, ties by the caller's id ascending.  The vertices most relaxations
 * reach then share cache sectors, which keeps more of the per-source distance
 * state in L2 during sssp_solve.  The paper has no such step: it only renames
 * vertices (a layout of the state in memory), and a solve on the result returns
 * exactly what it returns on g.
 *   g        : a graph in the caller's ids (g->ids == NULL), rows sorted as sssp_build_csr makes them
 *   row_ptr_out, col_out, w_out : device [V+1], [E], [E] out: the renumbered CSR (rows sorted)
 *   emap_out : device [E] out (may be NULL): index in g of stored edge k
 *   ids_out, slots_out : device [V] out: the sssp_graph ids / slots of the result
 *   ws       : device workspace >= sssp_layout_workspace_size(g); holds the status word
 * The result is the sssp_graph {V, E, row_ptr_out, col_out, w_out, wtype, partitions,
 * ids_out, slots_out}.
 */
sssp_status sssp_layout(const sssp_graph* g, uint32_t* row_ptr_out, uint32_t* col_out, void* w_out,
                        uint32_t* emap_out, uint32_t* ids_out, uint32_t* slots_out, void* ws, size_t ws_bytes,
                        sssp_stream_t stream);

/* ------------------------------------------------------------ K2 partition */

/*
 * 1D block partition (Sec. III.A, read as B = ceil(V/P), Pid(v) = floor(v/B)).
 *   bounds : device [P+1] out, bounds[p] = min(p*B, V)
 *   inter  : device [P] out (may be NULL), edges whose tail is in partition p and head is not --
 *            the "inter-edges" of Sec. III.D whose product with P is ToKa's message threshold.
 */
sssp_status sssp_partition(const sssp_graph* g, uint32_t* bounds, uint64_t* inter, sssp_stream_t stream);

/* ------------------------------------------------------------ K3 Trishla */

/*
 * Trishla (Sec. III.B, Algorithm 1): edge (u, v_j) is deleted when some
 * out-neighbour v_i of u has an edge (v_i, v_j) with
 *     w(u, v_j) > w(u, v_i) + w(v_i, v_j)      (strict; float32 sums rounded once).
 * mode 0 (local, the paper's E_i): v_i must be in u's partition.  mode 1
 * (global): any v_i.  Every test reads the unpruned graph, so the result does
 * not depend on evaluation order.
 *   keep    : device [E] out, 1 = kept, 0 = deleted
 *   witness : device [E] out (may be NULL), smallest such v_i, 0xFFFFFFFF for kept edges
 */
sssp_status sssp_prune(const sssp_graph* g, int32_t mode, uint8_t* keep, uint32_t* witness, sssp_stream_t stream);

/* Workspace bytes of sssp_compact. */
size_t sssp_compact_workspace_size(uint32_t V, uint32_t E);

/*
 * The graph without the edges with keep[e] == 0 (what the relaxation of
 * Sec. III.C then scans).  row_ptr_out device [V+1]; col_out, w_out,
 * emap_out device [E] (first *E_out valid); emap_out[k] = index in g of kept
 * edge k (may be NULL).  E_out device [1].
 */
sssp_status sssp_compact(const sssp_graph* g, const uint8_t* keep, uint32_t* row_ptr_out, uint32_t* col_out,
                         void* w_out, uint32_t* emap_out, uint32_t* E_out, void* ws, size_t ws_bytes,
                         sssp_stream_t stream);

/* --------------------------------------------------------- K0/K4 solve */

/* Workspace bytes of sssp_solve for graph g and S sources with options opt (may be NULL). */
size_t sssp_solve_workspace_size(const sssp_graph* g, uint32_t S, const sssp_options* opt);

/*
 * SP-Async (Sec. III.C, SP-Async and DIJKSTRA; Sec. III.D termination) for S
 * sources at once, each an independent problem on the same graph.
 *   sources : device [S] vertex ids (< V)
 *   dist    : device [S][V] out, uint32 or float32 per g->wtype
 *   pred    : device [S][V] out (may be NULL), canonical predecessor vertex
 *   ws      : device workspace >= sssp_solve_workspace_size(g, S, opt)
 * opt->policy chooses the frontier policy of a round (sssp_policy).
 * Launches an init kernel, one persistent cooperative relaxation kernel in
 * which each block owns (source, partition sub-block) units, and an unpack
 * kernel.  Needs every block co-resident; returns SSSP_EUNSUPPORTED if the
 * device cannot hold one block per unit... (it then reuses blocks over
 * several units, so it only fails if not even one block fits).
 */
sssp_status sssp_solve(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                       const sssp_options* opt, void* ws, size_t ws_bytes, sssp_stream_t stream);

/*
 * sssp_solve and sssp_prune in one pass, with the prune run on the solve's idle
 * time: Sec. III.B observes that a process that receives no message sits idle,
 * and spends that time finding edges that lie on no shortest path (Trishla,
 * Algorithm 1).  Here a block of the persistent solve that finds none of its
 * units queued runs Trishla chunks of g instead of waiting, and goes back to its
 * units after each chunk; the chunks left when the solve ends run in a launch
 * right after it.  The solve reads the unpruned g (pruned edges are never on a
 * shortest path, so its result is the same either way); the keep mask serves
 * later solves on the compacted graph (sssp_compact).
 *   g, sources, S, dist, pred, opt, ws, ws_bytes : as for sssp_solve
 *   mode, keep, witness : as for sssp_prune (keep device [E], witness device [E] or NULL);
 *                         the same values sssp_prune gives, on the CSR as stored
 */
sssp_status sssp_solve_prune(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                             int32_t mode, uint8_t* keep, uint32_t* witness, const sssp_options* opt, void* ws,
                             size_t ws_bytes, sssp_stream_t stream);

/*
 * Warm start (incremental SSSP; the paper has no such call): sssp_solve's result
 * on a graph after some edge weights fell or edges were added, computed from the
 * result before the change instead of from scratch.  Previous distances stay
 * upper bounds when weights only fall, and relaxing the tails of the changed
 * edges from them converges, as the label-correcting relaxation across
 * partitions of Sec. III.C does from any upper bounds, to the same distances and
 * canonical predecessors a fresh sssp_solve returns.
 *   g          : the graph after the change (same vertex ids; may be a different CSR)
 *   dist, pred : device [S][V] in/out: on entry a result of sssp_solve (or of this
 *                call) for S sources on the graph before the change, in the caller's
 *                ids; on exit the result on g.  pred must not be NULL.
 *   tails      : device [n_tails] caller's ids of the tails of every edge whose weight
 *                fell or that was added (repeats allowed); n_tails = 0 returns the input
 *   opt, ws    : as for sssp_solve (ws >= sssp_solve_workspace_size(g, S, opt))
 * A weight that rose is not allowed: the relaxation never raises a distance, so the
 * result would keep the old, now too small, value.  Bad tail ids end with SSSP_EINVAL
 * on the device status.
 */
sssp_status sssp_update(const sssp_graph* g, uint32_t S, void* dist, uint32_t* pred, const uint32_t* tails,
                        uint32_t n_tails, const sssp_options* opt, void* ws, size_t ws_bytes, sssp_stream_t stream);

/*
 * Autotuner for sssp_solve (the paper has no tuner; its knobs are the process
 * count and the termination timeout).  Runs sssp_solve on (g, sources) with
 * candidate schedules and returns the fastest: for each frontier policy
 * RELATIVE, FIXED and NEAR_FAR the bucket width delta is searched over
 * {1/64 .. 4} x the mean of a sample of the weights (powers of two), and ALL
 * once; the best is refined at 3/4 and 3/2 of its delta; on a layout graph
 * hub_count over {256, 512, 1024} is tried with 1, 1.5, 2 and 3 times that
 * delta under RELATIVE, FIXED and NEAR_FAR; then tile over {1024, 2048, 4096},
 * then split over {1, 2, 4}, then tile once more if the split changed (split
 * only where ws is large enough).  The base options' policy and hub_count are
 * ignored.  Each candidate runs `trials` times (>= 1) after one
 * warm-up, timed with CUDA events on `stream`; candidates that fail are
 * skipped.  Synchronous.  Results do not depend on the schedule, so dist and
 * pred hold a valid solve afterwards.
 *   base : options to start from (may be NULL); best : out; best_ms : out (may be NULL)
 *   ws   : as for sssp_solve with `base` (and split up to 4 if it fits)
 */
sssp_status sssp_autotune(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                          void* ws, size_t ws_bytes, const sssp_options* base, uint32_t trials,
                          sssp_options* best, float* best_ms, sssp_stream_t stream);

/*
 * Synchronise `stream`, then return the status recorded on the device by the
 * last call that used workspace `ws` (and clear nothing).  stats (host, may
 * be NULL) receives that call's counters (zero for calls that keep none).
 */
sssp_status sssp_workspace_status(const void* ws, sssp_stream_t stream, sssp_stats* stats);

/* ------------------------------------------------------ no-allocation solve */

/* Bytes of the fixed device array that backs sssp_solve_noalloc (reserved on
 * every GPU that loads the library, until the process exits). */
#define SSSP_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * sssp_solve for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a convenience of the library.  Some callers, such as
 * a plugin or user-defined function inside a host application that owns every
 * device allocation and hands extensions only their input and output buffers,
 * have no way to provide sssp_solve's workspace.  This call takes its scratch
 * from a fixed array of SSSP_NOALLOC_SCRATCH_BYTES that the library reserves
 * on each device, so it allocates nothing.
 *   g, sources, S, dist, pred, opt : as for sssp_solve
 *   status_out : device [1] uint32 (may be NULL), receives the solve's device-side
 *                sssp_status, copied on `stream` after the solve
 * Returns SSSP_ENOMEM (nothing launched) if sssp_solve_workspace_size(g, S, opt)
 * exceeds SSSP_NOALLOC_SCRATCH_BYTES.  The first call on a device resolves the
 * array's address (cudaGetSymbolAddress, with that device current) and caches
 * it with the id of the device's current context; make it before any stream
 * capture.  A call that finds another context current (after cudaDeviceReset,
 * for instance) resolves the address again, so it too belongs outside a
 * capture.  All calls share the array, which keeps the last
 * call's contents (each call re-initialises what it reads): calls that overlap
 * on the GPU race and must be ordered by the caller.
 */
sssp_status sssp_solve_noalloc(const sssp_graph* g, const uint32_t* sources, uint32_t S, void* dist, uint32_t* pred,
                               const sssp_options* opt, uint32_t* status_out, sssp_stream_t stream);

/* ------------------------------------------------------- multi-GPU sharding */

/*
 * Host-only (no device work, no stream): split independent problems across
 * n_ranks processes, one per GPU, by their estimated cost.  The paper's only
 * parallel strategy is the domain split over processes (Sec. III.A); for
 * independent problems (the sources of a multi-source solve, the (graph,
 * source) problems of a batch) the split needs no exchange at all, so each
 * rank calls this with the same arguments, gets the same answer and solves
 * its own problems.  Longest-processing-time-first: problems in decreasing
 * cost (ties by index) each go to the rank with the least total cost so far
 * (ties by lowest rank).  The largest total is then at most (4/3 - 1/(3 n_ranks))
 * times the best possible, and at most the mean total plus the largest cost.
 *   cost    : host [n_problems] estimated cost of each problem (for example the
 *             edges of its graph: a solve scans every edge it reaches)
 *   rank_of : host [n_problems] out, the rank (< n_ranks) that solves each problem
 *   load    : host [n_ranks] out (may be NULL), total cost given to each rank
 * Returns SSSP_EINVAL for n_ranks == 0 or NULL arrays (with n_problems > 0).
 */
sssp_status sssp_shard_problems(uint32_t n_problems, const uint64_t* cost, uint32_t n_ranks, uint32_t* rank_of,
                                uint64_t* load);

/* ------------------------------------------------------------ K5 batched */

/* One graph of a batch: its CSR lives inside shared concatenated arrays. */
typedef struct {
    uint64_t row_off;  /* offset of this graph's V+1 row_ptr entries in the concatenated row_ptr */
    uint64_t edge_off; /* offset of this graph's first edge in the concatenated col / w */
    uint32_t V;        /* vertices (row_ptr values are relative to edge_off) */
    uint32_t E;        /* edges */
} sssp_batch_graph;

/* A batch of independent problems (graph, source) over several graphs. */
typedef struct {
    uint32_t n_graphs;
    uint32_t n_problems;
    const sssp_batch_graph* graphs; /* host [n_graphs] */
    const uint32_t* prob_graph;     /* host [n_problems], graph index of each problem */
    const uint32_t* prob_source;    /* host [n_problems], source (graph-local id) */
    const uint32_t* row_ptr;        /* device, concatenated */
    const uint32_t* col;            /* device, concatenated, graph-local ids */
    const void* w;                  /* device, concatenated */
    int32_t wtype;
    void* dist;                     /* device out: problem i's V_g values start at out_off(i) = sum_{j<i} V_{graph(j)} */
    uint32_t* pred;                 /* device out, same layout (may be NULL) */
} sssp_batch;

/* Workspace bytes of the batched solve. */
size_t sssp_batch_workspace_size(const sssp_batch* b, const sssp_options* opt);

/*
 * Solve every problem of the batch in one persistent launch: blocks pull
 * problems from a device work queue (largest graphs first) and each solves
 * its problem alone -- init, Delta-ordered relaxation over the whole graph
 * (one partition), unpack -- with no message traffic between blocks.
 * Uploads the problem tables (host arrays) into ws on `stream` and waits for
 * that copy, then launches: unlike the other solve calls this one blocks the
 * host until the upload is done, and it cannot be captured into a CUDA graph
 * (the wait is not a stream operation).  The plan calls below upload once at
 * creation and replay with no host work, so they are the path to use inside a
 * capture or a loop.
 */
sssp_status sssp_solve_batched(const sssp_batch* b, const sssp_options* opt, void* ws, size_t ws_bytes,
                               sssp_stream_t stream);

/* A batched solve captured once into a CUDA graph and replayed. */
typedef struct sssp_batch_plan sssp_batch_plan;

/* Upload the tables, capture [counter reset, persistent kernel] into a CUDA
 * graph on `stream` and instantiate it.  The plan keeps b's device pointers
 * and ws; they must stay valid until sssp_batch_plan_destroy. Synchronous. */
sssp_status sssp_batch_plan_create(const sssp_batch* b, const sssp_options* opt, void* ws, size_t ws_bytes,
                                   sssp_stream_t stream, sssp_batch_plan** plan);
/* Replay the captured graph on `stream` (asynchronous). */
sssp_status sssp_batch_plan_launch(sssp_batch_plan* plan, sssp_stream_t stream);
void sssp_batch_plan_destroy(sssp_batch_plan* plan);

/* -------------------------------------------------------------- K6 backward */

size_t sssp_backward_workspace_size(uint32_t V, uint32_t E, uint32_t S);

/*
 * Gradient of L = sum_s sum_v grad_dist[s][v] * dist_s(v) with respect to
 * the edge weights (the paper has no gradients: dist_s(v) is the sum of the
 * weights on the tree path to v, so dL/dw(e) sums grad_dist over the subtree
 * below every tree edge e).  The upstream gradient is carried up each
 * predecessor tree, children before parents (a reverse topological order of
 * the tree, of which decreasing distance is one), accumulated in float64.
 *   pred      : device [S][V] canonical predecessors from sssp_solve
 *   grad_dist : device [S][V] float32 (values at unreachable vertices are ignored)
 * The distances themselves are not an argument: the predecessor tree alone
 * fixes which edges lie on each vertex's path, and the walk from every vertex
 * up to its source visits children before parents without sorting by distance
 * (an unreachable vertex, pred == 0xFFFFFFFF and not a source, starts no walk).
 *   grad_w    : device [E] float32 out, CSR edge order, summed over the S sources;
 *               non-tree edges get 0
 */
sssp_status sssp_backward(const sssp_graph* g, uint32_t S, const uint32_t* pred, const float* grad_dist,
                          float* grad_w, void* ws, size_t ws_bytes, sssp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SSSP_H */
