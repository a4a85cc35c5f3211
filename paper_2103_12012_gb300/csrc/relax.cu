// K0 init (fresh or warm) / K4 persistent relaxation / K5 batched relaxation / unpack.
//
// The SP-Async loop of Sec. III.C on one GPU.  Vertices are split into
// units: a unit is one sub-block of one partition (Sec. III.A 1D block
// partitioning, sub-divided `split` ways) for one source.  Each unit has one
// owner thread block (unit b, b + grid, ...), which serves its dirty units in
// source order.  Per source the device state is
//   packed[v] : 64-bit word (dist << 32 | label), lowered only by atomicMin;
//               dist is the uint32 distance or the bits of a non-negative
//               float32 distance, whose unsigned order is the numeric order;
//               label is the predecessor's id in the caller's numbering.
//   bitmap[v] : 1 bit per vertex, the inbox: set when v's distance dropped
//               and v must be (re)processed (Alg. 2 pq.push / Alg. 3 push or
//               send_msg), cleared by the owner when it takes v.
//   dirty[q]  : a unit's doorbell, rung after new bits land in its range.
// A round of a unit (Alg. 2 recv_msgs + DIJKSTRA, bucketed):
//   A  enumerate the unit's queued vertices (warp-cooperative over the inbox
//      words), read their distances, find the minimum dmin, and keep those
//      below (running minimum + delta), a superset of the bucket;
//   B  select from them the ones with dist < dmin + delta (the near bucket,
//      an approximation of Dijkstra's pop order inside the partition), at
//      most `tile` of them;
//   C  take them: clear their inbox bits (acquire);
//   D  re-read their distances and CSR row extents; prefix-sum the degrees;
//   E  relax every out-edge of the taken vertices with the whole block:
//      cand = d(u)+w(u,v); if it beats the target's distance (read first),
//      atomicMin the packed word with (cand, label(u)); if that lowered the
//      distance, set v's inbox bit after a release fence -- a message (Alg. 3
//      send_msg) when v is in another unit; a vertex of this unit that falls
//      below the bucket bound goes to a shared-memory queue instead and is
//      relaxed by a sub-round of the same round (Dijkstra inside the unit).
//      A sub-round of at most one edge per thread (the wavefront of a
//      high-diameter graph) is latency-bound: there a queued vertex's row
//      extents are loaded alongside its atomic, its entry goes straight into
//      the other half of the selection arrays, a single warp scans the degrees
//      of up to 32 vertices, the read-first filter is dropped while most
//      relaxations of the block reach the atomic, and a thread's message is
//      sent at the start of the next sub-round (its atomic overlapping that
//      sub-round's loads) or, after the last one, before F;
//   F  settle the termination count and ring the doorbells of every unit
//      that received a new vertex (and this unit's own if vertices are left).
// Termination (Sec. III.D, the message counter of ToKa): `pending` counts
// queued vertices plus the reservations of rounds in flight.  A block takes a
// fixed reservation (more than a round can activate) when it picks a unit,
// before any of the round's bits can be visible, and returns it at the end of
// the round together with the vertices it took, adding the ones it activated.
// pending == 0 therefore means no queued and no in-flight work anywhere, and
// it can never rise again; every block then exits.  Every wait is bounded by a
// %globaltimer limit after which the block records SSSP_ETIMEOUT, raises the
// abort flag and returns.  A warm start packs a previous result instead of
// the INF words and queues the tails of the changed edges.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sssp {
namespace {

constexpr unsigned long long SRC_KEY = 0x00000000FFFFFFFFull;  // dist 0, pred NONE
constexpr uint64_t KERNEL_LIMIT_FACTOR = 3;  // whole-kernel wall-clock limit = 3 x idle limit
constexpr uint32_t MAX_SUBROUNDS = 256;       // local sub-rounds one round may run
constexpr uint32_t GATHER_MIN = 1024;          // queued vertices one scan can keep (at least)
constexpr int GATHER_G = 2;                   // queued vertices a lane enumerates and loads together
constexpr uint32_t IDLE_BACKOFF_MAX_NS = 1024;  // longest sleep of a block with no dirty unit
constexpr uint64_t PRUNE_IDLE_NS = 20000;      // idle this long before a block runs Trishla chunks
// batched distance buckets: BK_NB fine buckets of width delta (the current coarse bucket),
// BK_NC coarse buckets of width BK_NB * delta after it, then one overflow.  8 + 8 keeps a
// problem's bitmaps at 17 bits a vertex (half of 16 + 16, whose state in flight misses L2 more):
// the 512-graph batch 41.6 ms against 42.6 ms, each at its best delta.
constexpr uint32_t BK_NB = 8, BK_NC = 8, BK_OV = BK_NB + BK_NC, BK_SLOTS = BK_NB + BK_NC + 1;
// edges in flight per thread in phase E: 3, and 4 in the hub variant (layout graphs with hubs,
// whose hub rows take the consecutive-edge mode): R-MAT scale 22 7.03 against 7.14 ms, while 4
// everywhere would slow the grid (50.6 against 45.1 ms) and 2 slows both
constexpr int EDGE_BATCH = 3;
constexpr int EDGE_BATCH_HUBS = 4;
constexpr uint32_t MSG_CAP = 64;             // messages one warp can hold (msg_buffer <= 32, plus one batch of 32)
// Termination counts a round reserves before any of its inbox bits can be visible.  A round
// runs at most MAX_SUBROUNDS sub-rounds; a sub-round relaxes the edges of distinct vertices,
// fewer than 2^32 (E is 32-bit), and turns on at most one inbox bit per relaxed edge, so a
// round's activations stay below MAX_SUBROUNDS * 2^32 <= the reserve.  With fewer than 2^22
// blocks in flight the 64-bit count cannot wrap.
constexpr unsigned long long ROUND_RESERVE = 1ull << 41;
static_assert(ROUND_RESERVE >= (unsigned long long)MAX_SUBROUNDS << 32, "reserve covers a round's activations");

// release ordering for the writes before it (an inbox bit after its lowered word)
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint32_t atom_and_acquire(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acquire.gpu.global.and.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Whole-warp reductions: one redux.sync (RX) or five dependent shuffles.  The persistent solve
// takes redux.sync (a small sub-round runs several of them between its barriers: grid 4096^2
// 48.5 against 49.3 ms); the batched kernel keeps the shuffles, which leave it fewer spills
// (47.0 against 47.2 ms on the 512-graph batch).
template <bool RX = true>
__device__ __forceinline__ uint32_t warp_min(uint32_t x) {
    if constexpr (RX) return __reduce_min_sync(0xFFFFFFFFu, x);
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
    return x;
}

template <bool RX = true>
__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
    if constexpr (RX) return __reduce_add_sync(0xFFFFFFFFu, x);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// bits of inbox word `wd` that belong to vertices in [lo, hi)
__device__ __forceinline__ uint32_t range_mask(uint32_t wd, uint32_t lo, uint32_t hi) {
    const uint32_t base = wd * 32u;
    uint32_t m = 0xFFFFFFFFu;
    if (base < lo) m &= 0xFFFFFFFFu << (lo - base);
    if (base + 32u > hi) m &= 0xFFFFFFFFu >> (base + 32u - hi);
    return m;
}

// In-place exclusive scan of a[0..n) in shared memory by the whole block;
// returns the total.  wsum: 32 words of shared scratch.
__device__ __forceinline__ uint32_t warp_scan_incl(uint32_t x, uint32_t lane) {
#pragma unroll
    for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// The vertex of the i-th set bit (i < the warp's total) of the 32 inbox words
// wb .. wb+31 a warp holds, one per lane: `bits` the lane's word, `incl` the
// inclusive prefix of the popcounts.  Binary lifting finds the word over the
// lanes' prefixes, then the bit over the word's prefix popcounts.
__device__ __forceinline__ uint32_t nth_queued(uint32_t wb, uint32_t bits, uint32_t incl, uint32_t i) {
    uint32_t w = 0;
#pragma unroll
    for (uint32_t s = 16; s; s >>= 1)
        if (__shfl_sync(0xFFFFFFFFu, incl, w + s - 1u) <= i) w += s;
    const uint32_t wbits = __shfl_sync(0xFFFFFFFFu, bits, w);
    const uint32_t r = i - (__shfl_sync(0xFFFFFFFFu, incl, w) - __popc(wbits));
    uint32_t p = 0;  // largest p with fewer than r+1 set bits below it
#pragma unroll
    for (uint32_t s = 16; s; s >>= 1)
        if ((uint32_t)__popc(wbits & ((1u << (p + s)) - 1u)) <= r) p += s;
    return (wb + w) * 32u + p;
}

// A slot of a shared list for each lane with `take` (one shared atomic per warp);
// NONE for the others.
__device__ __forceinline__ uint32_t warp_slot(bool take, uint32_t* count, uint32_t lane) {
    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, take);
    if (!ball) return NONE;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(count, (uint32_t)__popc(ball));
    base = __shfl_sync(0xFFFFFFFFu, base, 0) + (uint32_t)__popc(ball & ((1u << lane) - 1u));
    return take ? base : NONE;
}

// Appends v to list[0, cap) for the lanes with `take` (one shared atomic per warp).
__device__ __forceinline__ void warp_append(bool take, uint32_t v, uint32_t* list, uint32_t* count, uint32_t cap,
                                            uint32_t lane) {
    const uint32_t ball = __ballot_sync(0xFFFFFFFFu, take);
    if (!ball) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(count, (uint32_t)__popc(ball));
    base = __shfl_sync(0xFFFFFFFFu, base, 0) + (uint32_t)__popc(ball & ((1u << lane) - 1u));
    if (take && base < cap) list[base] = v;
}

__device__ uint32_t block_scan_excl(uint32_t* a, uint32_t n, uint32_t* wsum) {
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5, nw = T >> 5;
    const uint32_t chunk = (n + T - 1u) / T;
    const uint32_t beg = min(tid * chunk, n), end = min(beg + chunk, n);
    uint32_t s = 0;
    for (uint32_t i = beg; i < end; ++i) s += a[i];
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31u) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < nw ? wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if ((int)lane >= o) t += y;
        }
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    uint32_t base = (wid ? wsum[wid - 1] : 0u) + x - s;
    for (uint32_t i = beg; i < end; ++i) {
        uint32_t v = a[i];
        a[i] = base;
        base += v;
    }
    const uint32_t total = wsum[nw - 1];
    __syncthreads();
    return total;
}

// Bucket bound for a round: dmin + delta, at least one step above dmin,
// saturating to "everything finite".
template <class W>
__device__ __forceinline__ uint32_t bucket_bound(uint32_t dmin, uint32_t delta) {
    uint32_t t;
    if (!W::add(dmin, delta, t)) return 0xFFFFFFFFu;
    return t > dmin ? t : dmin + 1u;
}

// Bound of a round's bucket under the chosen frontier policy (every policy gives the same
// result; they differ in how many vertices a round takes).  Non-decreasing in dmin and above
// it, so a bound computed from a running minimum is never below the final one.
//   RELATIVE   dmin + delta
//   FIXED      the end of the fixed width-delta bucket holding dmin (Delta-stepping's buckets)
//   NEAR_FAR   the unit's split point nf while dmin lies below it, else dmin + delta (the round
//              then moves the split there)
//   ALL        every queued vertex (asynchronous Bellman-Ford inside the partition)
template <class W>
__device__ __forceinline__ uint32_t policy_bound(uint32_t dmin, uint32_t delta, uint32_t policy, uint32_t nf) {
    switch (policy) {
        case SSSP_POLICY_FIXED: return W::bucket_end(dmin, delta);
        case SSSP_POLICY_NEAR_FAR: return dmin < nf ? nf : bucket_bound<W>(dmin, delta);
        case SSSP_POLICY_ALL: return 0xFFFFFFFFu;
        default: return bucket_bound<W>(dmin, delta);
    }
}

struct Scalars {
    uint32_t cnt, nlist, dmin, nsel, nclaim, bad, te;
    uint32_t nf;  // near-far policy: this unit's split point at the start of the round
    unsigned long long act;  // inbox bits this round turned on (64-bit: see ROUND_RESERVE)
    uint32_t nlq[2];  // local-queue counts of even and odd sub-rounds (a small sub-round ends
                      // without the barrier after which one counter could be reset for the next)
    // batched buckets: current coarse bucket (absolute), current fine slot, least coarse
    // bucket in the overflow (a lower bound), this round's operation and slot, and the set
    // bits of each slot (fine, coarse, overflow)
    uint32_t bk_k0, bk_f, bk_ovmin, bk_op, bk_slot, bk_cnt[BK_SLOTS];
    int pick;
    unsigned long long prob;
    // thread 0's scheduling state (static mode), here rather than in every thread's registers
    uint32_t backoff;
    unsigned long long idle_start, t_begin;
    uint32_t prune_done;  // prune while idle: the job's chunks have all been handed out
    uint32_t prune_go;    // prune while idle: this pass runs a chunk (set by the pick)
};

// Block statistics in shared memory, in sssp_stats order (idle time in ns until
// the flush): kept there rather than in registers every thread would carry.
enum : int { ST_EDGES, ST_ATOMICS, ST_IMPROVED, ST_ACTS, ST_ROUNDS, ST_VERTS, ST_REMOTE, ST_IDLE, ST_PRUNE, ST_N };

// Per-round view of one problem (one source on one graph).
struct Ctx {
    const uint32_t* row_ptr;
    const uint32_t* col;
    const uint32_t* w;
    const uint32_t* ids;  // stored vertex -> caller's id, the predecessor label (NULL: identity)
    uint32_t V;
    unsigned long long* packed;
    uint32_t* bitmap;
    WsHeader* hdr;
    uint32_t delta, tile, gcap;
    uint32_t policy;  // SSSP_POLICY_* (static mode; the batched kernel has its own buckets)
    uint32_t msg_buffer;  // 0: direct messages; k: a warp pushes its held messages out at k (static mode)
    uint32_t hub_count, hub_delta, hub_mid;  // static mode, layout graphs: hubs per partition, bucket widths
    // static-ownership mode only
    uint32_t* dirty;  // this source's unit doorbells
    uint32_t* nf;     // this source's near-far split point per unit (owner block only)
    uint32_t B, Bq, split, Qw;
    uint32_t words;  // batched buckets: inbox words of one bucket bitmap
};

struct Smem {
    uint32_t* list_v;   // [gcap]  A: queued ids;       D/E: row start of taken vertex
    uint32_t* list_d;   // [gcap]  A: queued distances; D/E: distance of taken vertex
    uint32_t* sel_v;    // [tile]  taken vertex ids
    uint32_t* sel_pref; // [tile+1] degree prefix sums
    uint32_t* lq;       // [tile]  vertices of this unit lowered below the bucket bound (next sub-round)
    uint32_t* touched;  // [Qw] units that got a new queued vertex this round (static mode)
    uint32_t* msg;      // [warps][MSG_CAP] held messages (message buffering only, else NULL)
    uint32_t* wsum;     // [32]
    Scalars* sc;
    unsigned long long* st;  // [ST_N] block statistics
};

// A new inbox bit for v: one activation, and in static mode a doorbell for v's unit.
template <bool STATIC>
__device__ __forceinline__ void inbox_count(const Ctx& c, uint32_t v, uint32_t my_q, const Smem& sm, uint32_t& lact,
                                            uint32_t& n_rem) {
    ++lact;
    if (STATIC) {
        const uint32_t p = v / c.B;
        const uint32_t q = p * c.split + (v - p * c.B) / c.Bq;
        if (q != my_q) ++n_rem;
        atomicOr(&sm.touched[q >> 5], 1u << (q & 31u));
    }
}

// Sets v's inbox bit (the caller has fenced the lowered word before it); a new bit
// counts as an activation and, in static mode, marks v's unit for a doorbell.
template <bool STATIC>
__device__ __forceinline__ void inbox_set(const Ctx& c, uint32_t v, uint32_t my_q, const Smem& sm, uint32_t& lact,
                                          uint32_t& n_rem) {
    const uint32_t bit = 1u << (v & 31u);
    if (atomicOr(&c.bitmap[v >> 5], bit) & bit) return;
    inbox_count<STATIC>(c, v, my_q, sm, lact, n_rem);
}

// Batched buckets: files v (distance d, never below the current fine bucket bkb) in its
// fine bucket, its coarse bucket or the overflow; a new bit counts as an activation.
template <class W>
__device__ __forceinline__ void bucket_file(const Ctx& c, uint32_t v, uint32_t d, uint32_t bkb, Scalars& sc,
                                            uint32_t& lact) {
    const uint32_t bit = 1u << (v & 31u);
    const uint32_t b = W::bucket(d, c.delta);
    const uint32_t kc = b / BK_NB, k0 = bkb / BK_NB;
    const uint32_t sl = kc == k0 ? b % BK_NB : kc <= k0 + BK_NC ? BK_NB + kc % BK_NC : BK_OV;
    if (!(atomicOr(&c.bitmap[(size_t)sl * c.words + (v >> 5)], bit) & bit)) {
        ++lact;
        atomicAdd(&sc.bk_cnt[sl], 1u);
    }
    if (sl == BK_OV) atomicMin(&sc.bk_ovmin, kc);
}

// One round over the unit owning vertices [lo, hi).  Returns the number of
// queued vertices the scan found (0 = the unit's inbox was empty).
template <class W, bool STATIC, bool BK, bool HELD = false, bool HUBS = false>
__device__ uint32_t relax_round(const Ctx& c, uint32_t lo, uint32_t hi, uint32_t my_q,
                                const Smem& sm) {
    static_assert(!(STATIC && BK), "distance buckets belong to the batched kernel");
    static_assert(!HELD || STATIC, "message buffering belongs to the persistent solve");
    constexpr int EB = HUBS ? EDGE_BATCH_HUBS : EDGE_BATCH;
    const uint32_t T = blockDim.x, tid = threadIdx.x, lane = tid & 31u;
    Scalars& sc = *sm.sc;
    if (tid == 0) {
        sc.cnt = 0;
        sc.nlist = 0;
        sc.dmin = 0xFFFFFFFFu;
        sc.nsel = 0;
        sc.nclaim = 0;
        sc.act = 0;
        sc.bad = 0;
        if (STATIC) sc.nf = c.policy == SSSP_POLICY_NEAR_FAR ? c.nf[my_q] : 0u;
        // (static mode: the pick reserved this round's termination counts)
    }
    __syncthreads();

    uint32_t found = 0, nsel = 0, te = 0, thr = 0, bkb = 0;
    // Hubs (on a layout graph the first hub_count stored vertices of each partition: its
    // highest-degree ones) are taken only below thr_hub, a bucket of a quarter of the width,
    // and the next 3 * hub_count only below thr_mid, half of it: a vertex processed before its
    // distance settles is processed again, and for these that costs long rows.
    // (the narrower bounds are formed on demand from the round's minimum in shared memory: they are
    // needed only for candidates and improved targets, and kept in registers they cost spills)
    auto lim = [&](uint32_t v) {
        if (!HUBS) return thr;
        const uint32_t off = v - (v / c.B) * c.B;
        if (off >= 4u * c.hub_count) return thr;
        return min(thr, bucket_bound<W>(sm.sc->dmin, off < c.hub_count ? c.hub_delta : c.hub_mid));
    };
    if constexpr (BK) {
        // ---- Distance buckets (batched: one block owns the whole problem, so every
        // producer is this block), a two-level radix structure: a vertex is queued in the
        // fine bucket (width delta) of its distance when that lies in the current coarse
        // bucket k0, else in coarse bucket k0+1 .. k0+BK_NC (width BK_NB * delta), else in
        // the overflow.  A round relaxes the lowest non-empty fine bucket; an exhausted
        // coarse bucket is split into the fine ones, the overflow moved in when its least
        // coarse bucket comes within reach.  So a queued vertex is read a few times in all
        // instead of once per round.  Relaxing fine bucket b only yields distances in
        // bucket b or later, so an entry whose vertex's distance has fallen into a finished
        // bucket is stale (the vertex was relaxed there) and is dropped.
        enum { OP_DONE, OP_PROCESS, OP_SPLIT, OP_FLUSH, OP_FLUSH_NEW };
        if (tid == 0) {
            uint32_t op = OP_DONE, slot = NONE;
            const uint32_t k0 = sc.bk_k0;
            if (sc.bk_cnt[BK_OV] && sc.bk_ovmin <= k0 + BK_NC) {
                op = OP_FLUSH;  // overflow entries that belong in the coarse window move in first
            } else {
                for (uint32_t f = sc.bk_f; f < BK_NB; ++f)
                    if (sc.bk_cnt[f]) {
                        op = OP_PROCESS;
                        slot = f;
                        sc.bk_f = f;
                        break;
                    }
                if (op == OP_DONE) {
                    for (uint32_t j = 1; j <= BK_NC; ++j)
                        if (sc.bk_cnt[BK_NB + (k0 + j) % BK_NC]) {
                            op = OP_SPLIT;
                            slot = k0 + j;  // the coarse bucket to split
                            break;
                        }
                }
                if (op == OP_DONE && sc.bk_cnt[BK_OV]) op = OP_FLUSH_NEW;
            }
            sc.bk_op = op;
            sc.bk_slot = slot;
        }
        __syncthreads();
        const uint32_t op = sc.bk_op, k0 = sc.bk_k0;
        uint32_t* const bmap = c.bitmap;
        auto slot_bm = [&](uint32_t sl) { return bmap + (size_t)sl * c.words; };
        auto for_each_set = [&](const uint32_t* bm, auto&& f) {  // warp-uniform calls f(ok, v)
            for (uint32_t wb = tid & ~31u; wb < c.words; wb += T) {
                const uint32_t wd = wb + lane;
                const uint32_t bits = wd < c.words ? __ldcg(&bm[wd]) : 0u;
                const uint32_t incl = warp_scan_incl((uint32_t)__popc(bits), lane);
                const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                for (uint32_t i0 = lane; i0 < total + lane; i0 += 32u)
                    f(i0 < total, nth_queued(wb, bits, incl, min(i0, total - 1u)));
            }
        };
        auto dist = [&](uint32_t v) { return (uint32_t)(__ldcg(&c.packed[v]) >> 32); };
        // move v (its bit set in slot `from`) to the slot of fine bucket b under current coarse
        // bucket `base`; false if it belongs where it is
        auto move = [&](uint32_t* from_bm, uint32_t from, uint32_t v, uint32_t b, uint32_t base) {
            const uint32_t kc = b / BK_NB;
            const uint32_t to = kc == base ? b % BK_NB : kc <= base + BK_NC ? BK_NB + kc % BK_NC : BK_OV;
            if (to == from) return false;
            const uint32_t bit = 1u << (v & 31u);
            atomicAnd(&from_bm[v >> 5], ~bit);
            if (!(atomicOr(&slot_bm(to)[v >> 5], bit) & bit)) atomicAdd(&sc.bk_cnt[to], 1u);
            if (to == BK_OV) atomicMin(&sc.bk_ovmin, kc);
            return true;
        };
        if (op == OP_PROCESS) {
            // take up to `tile` queued vertices of the fine bucket (A/B), then (C/D) claim them,
            // drop the stale ones, read distances and row extents
            found = 1;
            const uint32_t slot = sc.bk_slot;
            bkb = k0 * BK_NB + slot;
            uint32_t* const bm = slot_bm(slot);
            for_each_set(bm, [&](bool ok, uint32_t v) {
                const uint32_t k = warp_slot(ok, &sc.nsel, lane);
                if (k < c.tile) sm.sel_v[k] = v;
            });
            __syncthreads();
            nsel = min(sc.nsel, c.tile);
            uint32_t myproc = 0;
            for (uint32_t i = tid; i < nsel; i += T) {
                const uint32_t u = sm.sel_v[i];
                atomicAnd(&bm[u >> 5], ~(1u << (u & 31u)));
                const uint32_t du = dist(u);
                uint32_t deg = 0, beg = 0;
                if (W::bucket(du, c.delta) < bkb) {
                    sm.sel_v[i] = NONE;
                } else {
                    ++myproc;
                    beg = __ldg(&c.row_ptr[u]);
                    deg = __ldg(&c.row_ptr[u + 1]) - beg;
                }
                sm.list_d[i] = du;
                sm.list_v[i] = beg;
                sm.sel_pref[i] = deg;
            }
            myproc = warp_sum<!BK>(myproc);
            if (lane == 0 && myproc) atomicAdd(&sc.nclaim, myproc);
            if (tid == 0) sc.bk_cnt[slot] -= nsel;
        } else if (op == OP_SPLIT) {
            // the fine buckets are exhausted: the next non-empty coarse bucket becomes k0 and
            // is split into them (entries whose distance fell into a finished bucket leave)
            found = 1;
            const uint32_t kn = sc.bk_slot, from = BK_NB + kn % BK_NC;
            uint32_t* const bm = slot_bm(from);
            uint32_t gone = 0;
            for_each_set(bm, [&](bool ok, uint32_t v) {
                if (!ok) return;
                const uint32_t b = W::bucket(dist(v), c.delta);
                ++gone;
                if (b / BK_NB < kn)  // stale
                    atomicAnd(&bm[v >> 5], ~(1u << (v & 31u)));
                else
                    move(bm, from, v, b, kn);
            });
            gone = warp_sum<!BK>(gone);
            if (lane == 0 && gone) atomicSub(&sc.bk_cnt[from], gone);
            __syncthreads();
            if (tid == 0) {
                sc.bk_k0 = kn;
                sc.bk_f = 0;
            }
        } else if (op == OP_FLUSH || op == OP_FLUSH_NEW) {
            // move the overflow into the window; for OP_FLUSH_NEW (nothing else queued) the
            // new current coarse bucket is the least live one of the overflow
            found = 1;
            uint32_t* const ov = slot_bm(BK_OV);
            uint32_t base = k0;
            if (op == OP_FLUSH_NEW) {
                for_each_set(ov, [&](bool ok, uint32_t v) {
                    uint32_t d = ok ? dist(v) : 0xFFFFFFFFu;
                    if (ok && W::bucket(d, c.delta) / BK_NB <= k0) d = 0xFFFFFFFFu;  // stale
                    const uint32_t m = warp_min<!BK>(d);
                    if (lane == 0 && m != 0xFFFFFFFFu) atomicMin(&sc.dmin, m);
                });
                __syncthreads();
                if (sc.dmin != 0xFFFFFFFFu) base = W::bucket(sc.dmin, c.delta) / BK_NB;
            }
            if (tid == 0) sc.bk_ovmin = 0xFFFFFFFFu;
            __syncthreads();
            uint32_t gone = 0;
            for_each_set(ov, [&](bool ok, uint32_t v) {
                if (!ok) return;
                const uint32_t b = W::bucket(dist(v), c.delta);
                const uint32_t kc = b / BK_NB;
                if (kc <= k0) {  // stale: fallen into a finished coarse bucket
                    atomicAnd(&ov[v >> 5], ~(1u << (v & 31u)));
                    ++gone;
                } else if (move(ov, BK_OV, v, b, base)) {
                    ++gone;
                } else {
                    atomicMin(&sc.bk_ovmin, kc);  // stays in the overflow
                }
            });
            gone = warp_sum<!BK>(gone);
            if (lane == 0 && gone) atomicSub(&sc.bk_cnt[BK_OV], gone);
            __syncthreads();
            if (tid == 0 && op == OP_FLUSH_NEW) {
                sc.bk_k0 = base;
                sc.bk_f = 0;
            }
        }
    } else {
        // ---- A: scan the inbox: count the queued vertices, find their minimum distance
        // and keep the candidates for the near bucket.  Each warp takes 32 words; its
        // lanes enumerate the set bits by rank, GATHER_G each with their distance loads
        // in flight together.  The block minimum only falls as the scan goes on, so a
        // vertex at or above (running minimum + delta) can never enter the bucket: only
        // the ones below it are kept (a superset of the bucket, usually far smaller
        // than all queued vertices).
        const uint32_t wlo = lo >> 5, whi = (hi - 1u) >> 5;
        for (uint32_t wb = wlo + (tid & ~31u); wb <= whi; wb += T) {
            const uint32_t wd = wb + lane;
            const uint32_t bits = wd <= whi ? ld_relaxed(&c.bitmap[wd]) & range_mask(wd, lo, hi) : 0u;
            const uint32_t incl = warp_scan_incl((uint32_t)__popc(bits), lane);
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (total == 0) continue;
            if (lane == 0) atomicAdd(&sc.cnt, total);
            for (uint32_t i0 = lane; i0 < total + lane; i0 += 32u * GATHER_G) {  // warp-uniform trip count
                uint32_t vs[GATHER_G], ds[GATHER_G];
#pragma unroll
                for (int g = 0; g < GATHER_G; ++g)
                    vs[g] = nth_queued(wb, bits, incl, min(i0 + 32u * g, total - 1u));
                uint32_t bm = 0xFFFFFFFFu;
#pragma unroll
                for (int g = 0; g < GATHER_G; ++g) {
                    ds[g] = i0 + 32u * g < total ? (uint32_t)(__ldcg(&c.packed[vs[g]]) >> 32) : 0xFFFFFFFFu;
                    bm = min(bm, ds[g]);
                }
                bm = warp_min<!BK>(bm);  // lane 0's first element is valid: bm is a distance
                if (lane == 0) atomicMin(&sc.dmin, bm);
                const uint32_t bound =
                    policy_bound<W>(min(bm, *(volatile uint32_t*)&sc.dmin), c.delta, c.policy, sc.nf);
#pragma unroll
                for (int g = 0; g < GATHER_G; ++g) {
                    const uint32_t k = warp_slot(ds[g] < bound, &sc.nlist, lane);
                    if (k < c.gcap) {
                        sm.list_v[k] = vs[g];
                        sm.list_d[k] = ds[g];
                    }
                }
            }
        }
        __syncthreads();
        found = sc.cnt;
        if (found != 0) {
            thr = policy_bound<W>(sc.dmin, c.delta, c.policy, sc.nf);
            // near-far: the near set ran dry below the split, so the split moves up
            if (STATIC && tid == 0 && c.policy == SSSP_POLICY_NEAR_FAR && sc.dmin >= sc.nf) c.nf[my_q] = thr;
            const uint32_t nkept = sc.nlist;

            // ---- B: the near bucket, at most `tile` vertices: from the kept candidates,
            // or, when there were more of them than the list holds, by enumerating the
            // inbox again
            if (nkept <= c.gcap) {
                for (uint32_t i = tid; i < nkept + lane; i += T) {  // warp-uniform trip count
                    const bool take = i < nkept && sm.list_d[i] < lim(sm.list_v[i]);
                    warp_append(take, take ? sm.list_v[i] : 0u, sm.sel_v, &sc.nsel, c.tile, lane);
                }
            } else {
                for (uint32_t wb = wlo + (tid & ~31u); wb <= whi; wb += T) {
                    const uint32_t wd = wb + lane;
                    const uint32_t bits = wd <= whi ? ld_relaxed(&c.bitmap[wd]) & range_mask(wd, lo, hi) : 0u;
                    const uint32_t incl = warp_scan_incl((uint32_t)__popc(bits), lane);
                    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
                    for (uint32_t i0 = lane; i0 < total + lane; i0 += 32u * GATHER_G) {
                        uint32_t vs[GATHER_G], ds[GATHER_G];
#pragma unroll
                        for (int g = 0; g < GATHER_G; ++g)
                            vs[g] = nth_queued(wb, bits, incl, min(i0 + 32u * g, total - 1u));
#pragma unroll
                        for (int g = 0; g < GATHER_G; ++g)
                            ds[g] = i0 + 32u * g < total ? (uint32_t)(__ldcg(&c.packed[vs[g]]) >> 32) : 0xFFFFFFFFu;
#pragma unroll
                        for (int g = 0; g < GATHER_G; ++g)
                            warp_append(ds[g] < lim(vs[g]), vs[g], sm.sel_v, &sc.nsel, c.tile, lane);
                    }
                }
            }
            __syncthreads();
            nsel = min(sc.nsel, c.tile);

            // ---- C: take them off the inbox (acquire: the producers' packed-word
            // updates are visible to the reads below); D: distances and row extents
            uint32_t myclaim = 0;
            for (uint32_t i = tid; i < nsel; i += T) {
                uint32_t u = sm.sel_v[i];
                const uint32_t bit = 1u << (u & 31u);
                const uint32_t old = atom_and_acquire(&c.bitmap[u >> 5], ~bit);
                uint32_t deg = 0, beg = 0, du = 0;
                if (old & bit) {
                    ++myclaim;
                    du = (uint32_t)(__ldcg(&c.packed[u]) >> 32);
                    beg = __ldg(&c.row_ptr[u]);
                    deg = __ldg(&c.row_ptr[u + 1]) - beg;
                    if (c.ids) sm.sel_v[i] = __ldg(&c.ids[u]);  // from here on sel_v holds predecessor labels
                } else {
                    sm.sel_v[i] = NONE;
                }
                sm.list_d[i] = du;
                sm.list_v[i] = beg;
                sm.sel_pref[i] = deg;
            }
            myclaim = warp_sum<!BK>(myclaim);
            if (lane == 0 && myclaim) atomicAdd(&sc.nclaim, myclaim);
        }
    }
    __syncthreads();
    if (found != 0) {
        // Sub-rounds: a relaxation that lowers a vertex of this unit below the bucket
        // bound queues it in shared memory (lq) and the next sub-round relaxes it, with
        // no inbox bit and no rescan -- Dijkstra inside the partition (Alg. 3) until the
        // bucket is exhausted or MAX_SUBROUNDS is reached.  Everything in lq is covered by
        // this round's reservation; whatever is left in lq at the end gets inbox bits.
        // Small sub-rounds (below) alternate their entries between the lower and the
        // upper half of the selection arrays: `base` is where this sub-round's are.
        const uint32_t H = c.tile >> 1;
        uint32_t base = 0;
        // A small sub-round is a chain of dependent global accesses, and a message (an inbox
        // bit in another unit, or in this one when the local queue is full) would add two
        // more to the thread that sends it.  So a thread of a small sub-round keeps its one
        // message (dv) and sends it at the start of the next sub-round, where the atomic's
        // round trip overlaps that sub-round's own loads; what is left is sent before the
        // round settles its termination count.
        uint32_t dv = NONE;
        for (uint32_t sub = 0;; ++sub) {
            if (nsel <= 32u) {  // one warp's scan, one barrier
                if (tid < 32u) {
                    const uint32_t x = lane < nsel ? sm.sel_pref[base + lane] : 0u;
                    const uint32_t inc = warp_scan_incl(x, lane);
                    if (lane < nsel) sm.sel_pref[base + lane] = inc - x;
                    if (lane == 31u) {
                        sm.sel_pref[base + nsel] = inc;
                        sc.te = inc;
                        sc.nlq[sub & 1u] = 0;
                        sm.st[ST_EDGES] += inc;
                    }
                }
                __syncthreads();
                te = sc.te;
            } else {
                te = block_scan_excl(sm.sel_pref + base, nsel, sm.wsum);
                if (tid == 0) {
                    sm.sel_pref[base + nsel] = te;
                    sc.nlq[sub & 1u] = 0;
                    sm.st[ST_EDGES] += te;
                }
                __syncthreads();
            }
            const bool last = sub + 1u >= MAX_SUBROUNDS;
            const bool small = te <= T && nsel < H;
            if (!small && base) {
                // the general path reads its entries from the lower half
                for (uint32_t i = tid; i <= nsel; i += T) {
                    if (i < nsel) {
                        sm.sel_v[i] = sm.sel_v[H + i];
                        sm.list_d[i] = sm.list_d[H + i];
                        sm.list_v[i] = sm.list_v[H + i];
                    }
                    sm.sel_pref[i] = sm.sel_pref[H + i];
                }
                base = 0;
                __syncthreads();
            }

            // ---- E: relax all out-edges, edge-parallel.  Each thread keeps EB edges
            // (EDGE_BATCH; EDGE_BATCH_HUBS in the hub variant) in flight together: all CSR
            // loads, then all read-first filters, then all atomics.  Its edges are a
            // block-width apart (lanes read consecutive edges: coalesced across short rows)
            // unless the taken vertices average 32 edges or more (hubs), where a warp takes
            // consecutive edges, its lane l the ones 32 apart, and one search of the degree
            // prefix serves the lane's batch.  Row of edge k: the largest a < nsel with
            // sel_pref[a] <= k (binary lifting, the batch's searches interleaved).
            uint32_t lact = 0, bad = 0;
            uint32_t n_ai = 0, n_rem = 0;  // statistics: atomics | improved << 16, remote activations
            uint32_t d_old = 0, d_bit = 0, d_v = NONE;  // the message held over from the last sub-round
            if (STATIC && dv != NONE) {
                fence_acq_rel();  // its lowered word (an atomic that has returned) before its bit
                d_v = dv;
                dv = NONE;
                d_bit = 1u << (d_v & 31u);
                d_old = atomicOr(&c.bitmap[d_v >> 5], d_bit);  // the result is read at the end
            }
            const bool consec = te >= 32u * nsel;
            // The read-first filter adds an L2 round trip before each atomic.  A sub-round
            // of at most one edge per thread is latency-bound, so the persistent solve drops
            // the filter there while this block's relaxations mostly reach the atomic (at
            // least one atomic per four edges so far: wavefront graphs such as grids).
            const bool filt = BK || te > T || sm.st[ST_ATOMICS] * 4u < sm.st[ST_EDGES];
            // consecutive mode: a warp takes 32 * EB consecutive edges and lane l edges
            // l, l + 32, ... of them, so every load instruction reads 32 consecutive words (lane l
            // taking 3 adjacent edges spreads each load over 384 bytes: 1.5% slower on R-MAT)
            const uint32_t kstep = consec ? 32u : T;
            const uint32_t top = nsel > 1u ? 1u << (31 - __clz(nsel - 1u)) : 0u;
            // A sub-round of at most one edge per thread is a chain of dependent global
            // accesses.  There thread k takes edge k, and a vertex of this unit that it
            // lowers below the bound has its row extents and label loaded alongside the
            // atomic and goes straight into the other half of the selection arrays (fewer
            // than H entries each), so the next sub-round reads no global memory before its
            // relaxations.
            if (small) {
                const uint32_t nb = base ^ H;
                if (tid < te) {
                    uint32_t a = base;
                    for (uint32_t st = top; st; st >>= 1)
                        if (a + st < base + nsel && sm.sel_pref[a + st] <= tid) a += st;
                    const uint32_t e = sm.list_v[a] + (tid - sm.sel_pref[a]);
                    const uint32_t v = __ldg(&c.col[e]);
                    uint32_t cand = __ldg(&c.w[e]);
                    if (!W::weight_ok(cand) || v >= c.V) {
                        bad |= 1u;
                    } else if (!W::add(sm.list_d[a], cand, cand)) {
                        bad |= 2u;
                    } else {
                        const bool mine = !last && v >= lo && v < hi &&
                                          (BK ? W::bucket(cand, c.delta) == bkb : cand < lim(v));
                        uint32_t beg = 0, end = 0, lab = v;
                        if (mine) {
                            beg = __ldg(&c.row_ptr[v]);
                            end = __ldg(&c.row_ptr[v + 1]);
                            if (c.ids) lab = __ldg(&c.ids[v]);
                        }
                        const unsigned long long key = ((unsigned long long)cand << 32) | sm.sel_v[a];
                        if (key < (filt ? __ldcg(&c.packed[v]) : ~0ull)) {
                            n_ai += 1u;
                            const unsigned long long old = atomicMin(&c.packed[v], key);
                            if (key < old && (uint32_t)(old >> 32) > cand) {
                                n_ai += 1u << 16;
                                const uint32_t pos = mine ? atomicAdd(&sc.nlq[sub & 1u], 1u) : H;
                                if (pos + 1u < H) {
                                    sm.sel_v[nb + pos] = lab;
                                    sm.list_d[nb + pos] = cand;
                                    sm.list_v[nb + pos] = beg;
                                    sm.sel_pref[nb + pos] = end - beg;
                                } else if constexpr (BK) {
                                    bucket_file<W>(c, v, cand, bkb, sc, lact);
                                } else {
                                    dv = v;  // sent by the next sub-round (or after the last)
                                }
                            }
                        }
                    }
                }
            } else {
                // message buffering: this warp's held messages (count warp-uniform)
                constexpr bool held = HELD;
                uint32_t* const mbuf = held ? sm.msg + (tid >> 5) * MSG_CAP : nullptr;
                uint32_t mn = 0;
                auto push_out = [&]() {  // every lowered word of the warp, one fence, then the bits
                    __syncwarp();
                    __threadfence();
                    for (uint32_t i = lane; i < mn; i += 32u) inbox_set<STATIC>(c, mbuf[i], my_q, sm, lact, n_rem);
                    __syncwarp();
                    mn = 0;
                };
                // with held messages the warp's lanes stay together (ballots): the trip count follows
                // lane 0's first edge, and lanes past the end carry no edge
                const uint32_t kwarp0 = consec ? (tid & ~31u) * EB : (tid & ~31u);
                for (uint32_t k0 = consec ? (tid & ~31u) * EB + lane : tid, kw = kwarp0; (held ? kw : k0) < te;
                     k0 += EB * T, kw += EB * T) {
                    uint32_t vv[EB], cc[EB], aa[EB];
    #pragma unroll
                    for (int j = 0; j < EB; ++j) aa[j] = 0;
                    if (consec) {
                        for (uint32_t st = top; st; st >>= 1)
                            if (aa[0] + st < nsel && sm.sel_pref[aa[0] + st] <= k0) aa[0] += st;
    #pragma unroll
                        for (int j = 1; j < EB; ++j) {  // step over row ends; sel_pref[nsel] = te
                            uint32_t a = aa[j - 1];
                            while (a + 1u < nsel && sm.sel_pref[a + 1u] <= k0 + (uint32_t)j * kstep) ++a;
                            aa[j] = a;
                        }
                    } else {
                        for (uint32_t st = top; st; st >>= 1) {
    #pragma unroll
                            for (int j = 0; j < EB; ++j) {
                                const uint32_t m = aa[j] + st;
                                if (m < nsel && sm.sel_pref[m] <= k0 + (uint32_t)j * T) aa[j] = m;
                            }
                        }
                    }
    #pragma unroll
                    for (int j = 0; j < EB; ++j) {
                        const uint32_t k = k0 + (uint32_t)j * kstep;
                        vv[j] = NONE;
                        if (k < te) {
                            const uint32_t a = aa[j];
                            const uint32_t e = sm.list_v[a] + (k - sm.sel_pref[a]);
                            vv[j] = __ldg(&c.col[e]);
                            cc[j] = __ldg(&c.w[e]);  // the weight, until it becomes the candidate below
                        }
                    }
                    unsigned long long cur[EB];
    #pragma unroll
                    for (int j = 0; j < EB; ++j) {
                        cur[j] = 0;
                        if (vv[j] == NONE) continue;
                        if (!W::weight_ok(cc[j]) || vv[j] >= c.V) {
                            bad |= 1u;
                            vv[j] = NONE;
                            continue;
                        }
                        if (!W::add(sm.list_d[aa[j]], cc[j], cc[j])) {
                            bad |= 2u;
                            vv[j] = NONE;
                            continue;
                        }
                        // read-first filter: a stale (higher) value only lets a useless atomic through
                        cur[j] = filt ? __ldcg(&c.packed[vv[j]]) : ~0ull;
                    }
                    uint32_t improved = 0;
    #pragma unroll
                    for (int j = 0; j < EB; ++j) {
                        if (vv[j] == NONE) continue;
                        const unsigned long long key = ((unsigned long long)cc[j] << 32) | sm.sel_v[aa[j]];
                        if (key < cur[j]) {
                            n_ai += 1u;
                            const unsigned long long old = atomicMin(&c.packed[vv[j]], key);
                            if (key < old && (uint32_t)(old >> 32) > cc[j]) {
                                n_ai += 1u << 16;
                                // near and in this unit: relax it in the next sub-round
                                const bool near = BK ? W::bucket(cc[j], c.delta) == bkb : cc[j] < lim(vv[j]);
                                if (!last && vv[j] >= lo && vv[j] < hi && near) {
                                    const uint32_t pos = atomicAdd(&sc.nlq[sub & 1u], 1u);
                                    if (pos < c.tile) {
                                        sm.lq[pos] = vv[j];
                                        continue;
                                    }
                                }
                                improved |= 1u << j;
                            }
                        }
                    }
                    if (n_ai & 0x80008000u) {  // keep both 16-bit halves from overflowing
                        atomicAdd(&sm.st[ST_ATOMICS], (unsigned long long)(n_ai & 0xFFFFu));
                        atomicAdd(&sm.st[ST_IMPROVED], (unsigned long long)(n_ai >> 16));
                        n_ai = 0;
                    }
                    uint32_t msgs = 0;  // improved vertices of other units, held for a push-out
                    if (held && improved) {
    #pragma unroll
                        for (int j = 0; j < EB; ++j) {
                            if (!(improved & (1u << j))) continue;
                            const uint32_t p = vv[j] / c.B;
                            if (p * c.split + (vv[j] - p * c.B) / c.Bq != my_q) msgs |= 1u << j;
                        }
                        improved &= ~msgs;
                    }
                    if (improved) {
                        // every lowered word before any of this thread's inbox bits (release);
                        // with buckets the only reader is this block, after its barriers
                        if constexpr (!BK) __threadfence();
    #pragma unroll
                        for (int j = 0; j < EB; ++j) {
                            if (!(improved & (1u << j))) continue;
                            const uint32_t v = vv[j];
                            if constexpr (BK)
                                bucket_file<W>(c, v, cc[j], bkb, sc, lact);
                            else
                                inbox_set<STATIC>(c, v, my_q, sm, lact, n_rem);
                        }
                    }
                    if (held) {
    #pragma unroll
                        for (int j = 0; j < EB; ++j) {
                            const bool has = (msgs >> j) & 1u;
                            const uint32_t ball = __ballot_sync(0xFFFFFFFFu, has);
                            if (has) mbuf[mn + (uint32_t)__popc(ball & ((1u << lane) - 1u))] = vv[j];
                            mn += (uint32_t)__popc(ball);
                            if (mn >= c.msg_buffer) push_out();  // size criterion
                        }
                    }
                }
                if (held && mn) push_out();  // age criterion: the end of the sub-round
            }
            if (STATIC && d_v != NONE && !(d_old & d_bit)) inbox_count<STATIC>(c, d_v, my_q, sm, lact, n_rem);
            lact = warp_sum<!BK>(lact);
            bad = __reduce_or_sync(0xFFFFFFFFu, bad);
            {
                const uint32_t wa = warp_sum<!BK>(n_ai & 0xFFFFu), wi = warp_sum<!BK>(n_ai >> 16);
                const uint32_t wr = warp_sum<!BK>(n_rem);
                if (lane == 0) {
                    if (wa) atomicAdd(&sm.st[ST_ATOMICS], (unsigned long long)wa);
                    if (wi) atomicAdd(&sm.st[ST_IMPROVED], (unsigned long long)wi);
                    if (wr) atomicAdd(&sm.st[ST_REMOTE], (unsigned long long)wr);
                }
            }
            if (lane == 0) {
                if (lact) atomicAdd(&sc.act, (unsigned long long)lact);
                if (bad) atomicOr(&sc.bad, bad);
            }
            __syncthreads();
            const uint32_t nlq = min(sc.nlq[sub & 1u], small ? H - 1u : c.tile);
            if (nlq == 0) break;
            if (small) {  // the entries are in place already (as relaxed)
                if (tid == 0) sm.st[ST_VERTS] += nlq;
                nsel = nlq;
                base ^= H;
                continue;
            }
            // the next sub-round's entries: the queued local vertices with fresh distances
            for (uint32_t i = tid; i < nlq; i += T) {
                const uint32_t u = sm.lq[i];
                sm.sel_v[i] = c.ids ? __ldg(&c.ids[u]) : u;
                sm.list_d[i] = (uint32_t)(__ldcg(&c.packed[u]) >> 32);
                const uint32_t beg = __ldg(&c.row_ptr[u]);
                sm.list_v[i] = beg;
                sm.sel_pref[i] = __ldg(&c.row_ptr[u + 1]) - beg;
            }
            if (tid == 0) sm.st[ST_VERTS] += nlq;
            nsel = nlq;
            __syncthreads();
        }
        if (STATIC) {  // the messages of the last sub-round
            uint32_t lact = 0, n_rem = 0;
            if (dv != NONE) {
                fence_acq_rel();
                inbox_set<STATIC>(c, dv, my_q, sm, lact, n_rem);
            }
            lact = warp_sum<!BK>(lact);
            n_rem = warp_sum<!BK>(n_rem);
            if (lane == 0) {
                if (lact) atomicAdd(&sc.act, (unsigned long long)lact);
                if (n_rem) atomicAdd(&sm.st[ST_REMOTE], (unsigned long long)n_rem);
            }
            __syncthreads();
        }
    }

    // ---- F: settle the count, ring doorbells (warp 0)
    if (tid < 32) {
        if (STATIC) {
            if (tid == 0) {
                const unsigned long long d =
                    sc.act - ROUND_RESERVE - (unsigned long long)sc.nclaim;
                atomicAdd(&c.hdr->pending, d);  // two's complement: adds act, returns reserve and takes
            }
            __threadfence();  // new bits (set before the barrier above) before the doorbells
            for (uint32_t wq = tid; wq < c.Qw; wq += 32u) {
                uint32_t bits = sm.touched[wq];
                if (!bits) continue;
                sm.touched[wq] = 0;
                while (bits) {
                    const uint32_t b = __ffs(bits) - 1u;
                    bits &= bits - 1u;
                    st_relaxed(&c.dirty[wq * 32u + b], 1u);
                }
            }
            if (tid == 0 && found > sc.nclaim) st_relaxed(&c.dirty[my_q], 1u);  // more left in this unit
        }
        if (tid == 0 && found) {
            sm.st[ST_ROUNDS] += 1;
            sm.st[ST_VERTS] += sc.nclaim;
            sm.st[ST_ACTS] += sc.act;
            if (sc.bad & 1u) set_status(c.hdr, SSSP_EINVAL);
            if (sc.bad & 2u) set_status(c.hdr, SSSP_EOVERFLOW);
        }
    }
    __syncthreads();
    return found;
}

__host__ __device__ inline uint32_t gather_cap(uint32_t tile) { return tile > GATHER_MIN ? tile : GATHER_MIN; }

__device__ Smem carve(uint32_t* dsm, uint32_t tile, uint32_t Qw, uint32_t* wsum, Scalars* sc,
                      unsigned long long* st, bool msgs = false) {
    const uint32_t gcap = gather_cap(tile);
    Smem s;
    s.list_v = dsm;
    s.list_d = dsm + gcap;
    s.sel_v = dsm + 2 * gcap;
    s.sel_pref = s.sel_v + tile;
    s.lq = s.sel_pref + tile + 1;
    s.touched = s.lq + tile;
    s.msg = msgs ? s.touched + ((Qw + 3u) & ~3u) : nullptr;
    s.wsum = wsum;
    s.sc = sc;
    s.st = st;
    for (uint32_t i = threadIdx.x; i < ST_N; i += blockDim.x) st[i] = 0ull;
    (void)Qw;
    return s;
}

__device__ void flush_stats(WsHeader* h, const unsigned long long* st) {
    const uint32_t i = threadIdx.x;
    if (i < ST_N) {
        const unsigned long long x = i == ST_IDLE ? st[i] / 1000ull : st[i];
        if (x) atomicAdd(&h->stats[i], x);
    }
}

// ---------------------------------------------------------------- kernels

// K0: every packed word to INF, inboxes and doorbells to zero.
__global__ void k_init_fill(unsigned long long* packed, size_t n_packed, uint32_t* bitmap, size_t n_words,
                            uint32_t* dirty, size_t n_dirty) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    ulonglong2* p2 = reinterpret_cast<ulonglong2*>(packed);
    for (size_t j = i; j < n_packed / 2; j += stride) p2[j] = make_ulonglong2(INF_KEY, INF_KEY);
    if (i == 0 && (n_packed & 1)) packed[n_packed - 1] = INF_KEY;
    for (size_t j = i; j < n_words; j += stride) bitmap[j] = 0u;
    for (size_t j = i; j < n_dirty; j += stride) dirty[j] = 0u;
}

// K0: seed each source (Alg. 2: d(s) = 0, pq.push(s) by the owner of s).
__global__ void k_seed(SolveLaunch L) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0 && L.hold_pending) atomicAdd(&L.hdr->pending, 1ull);
    if (s >= L.S) return;
    uint32_t src = L.sources[s];
    if (src >= L.V) {
        set_status(L.hdr, SSSP_EINVAL);
        return;
    }
    if (L.slots) src = L.slots[src];  // caller's id -> stored vertex
    L.packed[(size_t)s * L.V + src] = SRC_KEY;
    atomicOr(&L.bitmap[(size_t)s * L.words + (src >> 5)], 1u << (src & 31u));
    const uint32_t p = src / L.B;
    const uint32_t q = p * L.split + (src - p * L.B) / L.Bq;
    atomicAdd(&L.hdr->pending, 1ull);
    __threadfence();
    L.dirty[(size_t)s * L.Q + q] = 1u;
}

// dist / pred in the caller's ids: element i of source s reads the packed word of
// stored vertex slots[i] (predecessor labels are caller's ids already).
// K0 (warm start): the packed words from a previous result, given in the caller's
// order (dist [S][V], pred [S][V]); an unreached vertex gets the INF word.
template <class W>
__global__ void k_warm_pack(size_t n, uint32_t V, const uint32_t* __restrict__ slots,
                            const uint32_t* __restrict__ dist, const uint32_t* __restrict__ pred,
                            unsigned long long* __restrict__ packed) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const size_t s = i / V, j = i - s * V;
        const size_t at = s * V + (slots ? __ldg(&slots[j]) : j);
        const uint32_t d = dist[i];
        packed[at] = d == W::inf_out() ? INF_KEY : ((unsigned long long)d << 32) | pred[i];
    }
}

// K0 (warm start): queue, in every source, the tails of the edges whose weight fell or
// that were added (a reached tail only: an unreached one relaxes nothing).  Relaxing
// them from the previous distances, which stay upper bounds when weights only fall,
// converges to the new result (label correcting, as the Bellman-Ford level of Sec. III.C).
__global__ void k_warm_seed(SolveLaunch L) {
    const size_t n = (size_t)L.S * L.n_tails;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gtid == 0 && L.hold_pending) atomicAdd(&L.hdr->pending, 1ull);
    for (size_t i = gtid; i < n; i += stride) {
        const uint32_t s = (uint32_t)(i / L.n_tails);
        const uint32_t t = L.warm_tails[i - (size_t)s * L.n_tails];
        if (t >= L.V) {
            set_status(L.hdr, SSSP_EINVAL);
            continue;
        }
        const uint32_t v = L.slots ? L.slots[t] : t;
        if (L.packed[(size_t)s * L.V + v] == INF_KEY) continue;
        const uint32_t bit = 1u << (v & 31u);
        if (atomicOr(&L.bitmap[(size_t)s * L.words + (v >> 5)], bit) & bit) continue;  // listed twice
        const uint32_t p = v / L.B;
        const uint32_t q = p * L.split + (v - p * L.B) / L.Bq;
        atomicAdd(&L.hdr->pending, 1ull);
        __threadfence();
        L.dirty[(size_t)s * L.Q + q] = 1u;
    }
}

template <class W>
__global__ void k_unpack(const unsigned long long* __restrict__ packed, size_t n, uint32_t V,
                         const uint32_t* __restrict__ slots, uint32_t* __restrict__ dist, uint32_t* __restrict__ pred) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        size_t at = i;
        if (slots) {
            const size_t s = i / V;
            at = s * V + __ldg(&slots[i - s * V]);
        }
        const unsigned long long k = packed[at];
        dist[i] = k == INF_KEY ? W::inf_out() : (uint32_t)(k >> 32);
        if (pred) pred[i] = k == INF_KEY ? NONE : (uint32_t)k;
    }
}

// K4: persistent, static ownership: block b owns units b, b+grid, b+2*grid, ...
// Four 512-thread blocks per SM: occupancy (2048 threads per SM) hides the
// memory latency of the relaxation better than more edges in flight per thread.
// PRUNE (sssp_solve_prune): a block that finds no dirty unit runs chunks of the Trishla job
// (each warp one chunk, claimed from the header's cursor) instead of sleeping -- the paper's
// use of the time processes spend waiting for messages (Sec. III.B) -- and goes back to its
// doorbells after each; the chunks left when the solve ends are run by a launch after it.
// HELD: message buffering (msg_buffer > 0); HUBS: hub widths (hub_count > 0 on a layout graph).
// Separate instantiations, so that the plain path keeps its registers.
template <class W, bool PRUNE, bool HELD, bool HUBS>
__global__ void __launch_bounds__(SOLVE_MAX_THREADS, 4) k_solve(SolveLaunch L) {
    extern __shared__ uint32_t dsm[];
    __shared__ uint32_t wsum[32];
    __shared__ Scalars sc;
    __shared__ unsigned long long st[ST_N];
    const uint32_t Qw = (L.Q + 31u) / 32u;
    const Smem sm = carve(dsm, L.tile, Qw, wsum, &sc, st, HELD);
    for (uint32_t i = threadIdx.x; i < Qw; i += blockDim.x) sm.touched[i] = 0u;
    __syncthreads();

    if (threadIdx.x == 0) {
        sc.backoff = 32;
        sc.idle_start = 0;
        sc.t_begin = globaltimer_ns();
        sc.prune_done = PRUNE ? 0u : 1u;
        sc.prune_go = 0u;
    }
    Ctx c;
    c.row_ptr = L.row_ptr;
    c.col = L.col;
    c.w = L.w;
    c.ids = L.ids;
    c.V = L.V;
    c.hdr = L.hdr;
    c.delta = L.delta_bits;
    c.tile = L.tile;
    c.gcap = gather_cap(L.tile);
    c.policy = L.policy;
    c.msg_buffer = L.msg_buffer;
    c.hub_count = L.hub_count;
    c.hub_delta = L.hub_delta_bits;
    c.hub_mid = L.hub_mid_bits;
    c.B = L.B;
    c.Bq = L.Bq;
    c.split = L.split;
    c.Qw = Qw;
    for (;;) {
        if (threadIdx.x < 32) {
            // warp 0 picks: lane 0 checks the limits, the lanes read the block's doorbells
            // together, and the lowest dirty unit (units in source order: a block serves
            // its lower sources first, so the state in use at any time belongs to few
            // sources) is taken with an exchange
            const uint32_t lane = threadIdx.x;
            const uint32_t U = L.S * L.Q;
            const uint32_t nu = blockIdx.x < U ? (U - 1u - blockIdx.x) / gridDim.x + 1u : 0u;
            int pick = -1;
            if (lane == 0) {
                if (ld_relaxed(&L.hdr->abort_flag)) {
                    pick = -2;
                } else if (globaltimer_ns() - sc.t_begin > KERNEL_LIMIT_FACTOR * L.timeout_ns) {
                    // whole-kernel limit: even a busy block cannot run unbounded
                    set_status(L.hdr, SSSP_ETIMEOUT);
                    atomicExch(&L.hdr->abort_flag, 1u);
                    pick = -2;
                }
            }
            pick = __shfl_sync(0xFFFFFFFFu, pick, 0);
            for (uint32_t j0 = 0; pick == -1 && j0 < nu; j0 += 32u) {
                const uint32_t uid = blockIdx.x + (j0 + lane) * gridDim.x;
                uint32_t ball = __ballot_sync(0xFFFFFFFFu, j0 + lane < nu && ld_relaxed(&L.dirty[uid]) != 0u);
                while (ball) {
                    const uint32_t f = __ffs(ball) - 1u;
                    uint32_t got = 0;
                    if (lane == f) got = atomicExch(&L.dirty[uid], 0u);
                    if (__shfl_sync(0xFFFFFFFFu, got, (int)f) != 0u) {
                        pick = (int)(blockIdx.x + (j0 + f) * gridDim.x);
                        break;
                    }
                    ball &= ball - 1u;
                }
            }
            if (lane == 0) {
                if (pick >= 0) {
                    // Reserve termination counts for the round before any of its inbox
                    // bits can be visible (a round activates at most one vertex per
                    // relaxed edge, fewer than ROUND_RESERVE); the same fence orders the
                    // doorbell before the inbox scan.
                    atomicAdd(&L.hdr->pending, ROUND_RESERVE);
                    __threadfence();
                    if (sc.idle_start) sm.st[ST_IDLE] += globaltimer_ns() - sc.idle_start;
                    sc.idle_start = 0;
                    sc.backoff = 32;
                } else if (pick == -1 && ld_relaxed(&L.hdr->pending) == 0ull) {
                    pick = -2;  // nothing queued, nothing in flight: terminated
                    if (sc.idle_start) sm.st[ST_IDLE] += globaltimer_ns() - sc.idle_start;
                } else if (pick == -1) {
                    const uint64_t now = globaltimer_ns();
                    if (sc.idle_start == 0) {
                        sc.idle_start = now;
                    } else if (now - sc.idle_start > L.timeout_ns) {
                        set_status(L.hdr, SSSP_ETIMEOUT);
                        atomicExch(&L.hdr->abort_flag, 1u);
                        pick = -2;
                    }
                    // a block idle for a while runs a Trishla chunk instead of sleeping
                    sc.prune_go = pick == -1 && !sc.prune_done && sc.idle_start &&
                                  now - sc.idle_start >= PRUNE_IDLE_NS;
                    if (pick == -1 && !sc.prune_go) {
                        __nanosleep(sc.backoff);
                        if (sc.backoff < IDLE_BACKOFF_MAX_NS) sc.backoff *= 2u;
                    }
                }
                sc.pick = pick;
            }
        }
        __syncthreads();
        const int pick = sc.pick;
        __syncthreads();
        if (pick == -2) break;
        if (pick < 0) {
            if constexpr (PRUNE) {
                if (sc.prune_go) {  // (written by the pick before the barrier above: the same in every thread)
                    // each warp one chunk, its light pairs only (the heavy ones wait for the launch after
                    // the solve), then back to the doorbells
                    const uint32_t lane = threadIdx.x & 31u;
                    unsigned long long ch = 0;
                    if (lane == 0) ch = atomicAdd(&L.hdr->work_next, 1ull);
                    ch = __shfl_sync(0xFFFFFFFFu, ch, 0);
                    if (ch < L.prune.nchunks) {
                        trishla_chunk<W>(L.prune, (uint32_t)ch, TRI_LIGHT);
                        if (lane == 0) atomicAdd(&sm.st[ST_PRUNE], 1ull);
                    } else if (lane == 0) {
                        sc.prune_done = 1u;
                    }
                    __syncthreads();  // (prune_done and prune_go are next touched by the pick)
                }
            }
            continue;
        }
        const uint32_t s = (uint32_t)pick / L.Q, q = (uint32_t)pick % L.Q;
        const uint32_t p = q / L.split, k = q % L.split;
        const uint32_t plo = p * L.B;
        const uint32_t phi = min(plo + L.B, L.V);
        const uint32_t lo = plo + k * L.Bq;
        const uint32_t hi = min(lo + L.Bq, phi);
        if (lo >= hi) {  // an empty sub-block is never dirty; return the reservation all the same
            if (threadIdx.x == 0) atomicAdd(&L.hdr->pending, 0ull - ROUND_RESERVE);
            continue;
        }
        c.packed = L.packed + (size_t)s * L.V;
        c.bitmap = L.bitmap + (size_t)s * L.words;
        c.dirty = L.dirty + (size_t)s * L.Q;
        c.nf = L.nfsplit + (size_t)s * L.Q;
        relax_round<W, true, false, HELD, HUBS>(c, lo, hi, q, sm);
    }
    __syncthreads();
    flush_stats(L.hdr, sm.st);
}

// K5: persistent, dynamic: blocks pull whole problems from a work queue.  Compiled for
// 2 x 1024 threads per SM (the register budget of 4 x 512): two 1024-thread blocks hold half the
// problems in flight, and so half the distance state competing for L2, with twice the threads on
// each problem's rounds (the 512-graph batch: 44.2 ms at tile 2048 against 47.0 ms with four
// 512-thread blocks at tile 1024).
template <class W>
__global__ void __launch_bounds__(BATCH_MAX_THREADS, 2) k_batched(BatchLaunch L) {
    extern __shared__ uint32_t dsm[];
    __shared__ uint32_t wsum[32];
    __shared__ Scalars sc;
    __shared__ unsigned long long st[ST_N];
    const Smem sm = carve(dsm, L.tile, 0u, wsum, &sc, st);
    Ctx c;
    c.hdr = L.hdr;
    c.delta = L.delta_bits;
    c.tile = L.tile;
    c.gcap = gather_cap(L.tile);
    c.dirty = nullptr;
    c.nf = nullptr;
    c.policy = SSSP_POLICY_RELATIVE;
    c.msg_buffer = 0;
    c.hub_count = 0;
    c.hub_delta = 0;
    c.hub_mid = 0;
    c.ids = nullptr;
    c.B = c.Bq = c.split = 1u;
    c.Qw = 0;
    const uint32_t T = blockDim.x, tid = threadIdx.x;
    const uint64_t t_begin = globaltimer_ns();
    for (;;) {
        if (tid == 0) {
            sc.prob = ld_relaxed(&L.hdr->abort_flag) ? ~0ull : atomicAdd(&L.hdr->work_next, 1ull);
        }
        __syncthreads();
        const unsigned long long pi = sc.prob;
        __syncthreads();
        if (pi >= L.n_problems) break;
        const BatchProblem P = L.probs[pi];
        if (P.V == 0) continue;
        c.row_ptr = L.row_ptr + P.row_off;
        c.col = L.col + P.edge_off;
        c.w = L.w + P.edge_off;
        c.V = P.V;
        c.packed = L.packed + P.out_off;
        const uint32_t words = (P.V + 31u) / 32u;
        c.words = words;
        c.bitmap = L.bitmap + (size_t)BK_SLOTS * P.bm_off;  // the problem's fine, coarse and overflow bitmaps
        for (uint32_t i = tid; i < P.V; i += T) c.packed[i] = INF_KEY;
        for (uint32_t i = tid; i < BK_SLOTS * words; i += T) c.bitmap[i] = 0u;
        if (tid < BK_SLOTS) sc.bk_cnt[tid] = 0u;
        __syncthreads();
        if (tid == 0) {
            sc.bk_k0 = 0;
            sc.bk_f = 0;
            sc.bk_ovmin = 0xFFFFFFFFu;
            if (P.src < P.V) {
                c.packed[P.src] = SRC_KEY;
                c.bitmap[P.src >> 5] = 1u << (P.src & 31u);  // fine bucket 0
                sc.bk_cnt[0] = 1u;
            } else {
                set_status(L.hdr, SSSP_EINVAL);
            }
        }
        __syncthreads();
        for (;;) {
            const uint32_t found = relax_round<W, false, true>(c, 0u, P.V, 0u, sm);
            if (tid == 0) {
                int go = found != 0u;
                if (go && globaltimer_ns() - t_begin > KERNEL_LIMIT_FACTOR * L.timeout_ns) {
                    set_status(L.hdr, SSSP_ETIMEOUT);
                    atomicExch(&L.hdr->abort_flag, 1u);
                    go = 0;
                }
                sc.pick = go;
            }
            __syncthreads();
            const int go = sc.pick;
            __syncthreads();
            if (!go) break;
        }
        uint32_t* dist = L.dist + P.out_off;
        uint32_t* pred = L.pred ? L.pred + P.out_off : nullptr;
        for (uint32_t i = tid; i < P.V; i += T) {
            const unsigned long long k = ld_relaxed(&c.packed[i]);
            dist[i] = k == INF_KEY ? W::inf_out() : (uint32_t)(k >> 32);
            if (pred) pred[i] = k == INF_KEY ? NONE : (uint32_t)k;
        }
        __syncthreads();
    }
    __syncthreads();
    flush_stats(L.hdr, sm.st);
}

template <class K>
cudaError_t set_smem(K kernel, size_t smem) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

template <class W>
const void* solve_kernel(bool prune, bool held, bool hubs) {
    if (hubs) {
        if (held) return prune ? (const void*)k_solve<W, true, true, true> : (const void*)k_solve<W, false, true, true>;
        return prune ? (const void*)k_solve<W, true, false, true> : (const void*)k_solve<W, false, false, true>;
    }
    if (held) return prune ? (const void*)k_solve<W, true, true, false> : (const void*)k_solve<W, false, true, false>;
    return prune ? (const void*)k_solve<W, true, false, false> : (const void*)k_solve<W, false, false, false>;
}

size_t relax_smem_bytes(uint32_t tile, uint32_t Q, bool msgs) {
    size_t b = (size_t)(2u * gather_cap(tile) + 3u * tile + 1u) * 4u;
    if (!msgs) return b + (size_t)((Q + 31u) / 32u) * 4u;
    return b + (size_t)((((Q + 31u) / 32u) + 3u) & ~3u) * 4u + (size_t)(SOLVE_MAX_THREADS / 32u) * MSG_CAP * 4u;
}

cudaError_t relax_max_blocks_per_sm(int wtype, uint32_t threads, uint32_t tile, uint32_t Q, int* out, bool prune,
                                    bool msgs, bool hubs) {
    const size_t smem = relax_smem_bytes(tile, Q, msgs);
    const void* k = wtype == SSSP_W_F32 ? solve_kernel<WF32>(prune, msgs, hubs) : solve_kernel<WU32>(prune, msgs, hubs);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k, (int)threads, smem);
}

cudaError_t launch_solve(const SolveLaunch& L, cudaStream_t st) {
    cudaError_t e;
    const size_t n_packed = (size_t)L.S * L.V;
    const size_t n_words = (size_t)L.S * L.words;
    const size_t n_dirty = (size_t)L.S * L.Q;
    if ((e = cudaMemsetAsync(L.hdr, 0, WS_HEADER_BYTES, st)) != cudaSuccess) return e;  // (also the prune cursor)
    if ((e = cudaMemsetAsync(L.nfsplit, 0, 4 * n_dirty, st)) != cudaSuccess) return e;
    if (L.prune_on && (e = trishla_init(L.prune, st)) != cudaSuccess) return e;
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t want = (n_packed / 2 + 255) / 256;
        const unsigned blocks = (unsigned)std::min<size_t>(std::max<size_t>(want, 1), (size_t)sms * 8);
        if (L.warm) {
            if ((e = cudaMemsetAsync(L.bitmap, 0, 4 * n_words, st)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(L.dirty, 0, 4 * n_dirty, st)) != cudaSuccess) return e;
            if (L.wtype == SSSP_W_F32)
                k_warm_pack<WF32><<<blocks, 256, 0, st>>>(n_packed, L.V, L.slots, L.dist, L.pred, L.packed);
            else
                k_warm_pack<WU32><<<blocks, 256, 0, st>>>(n_packed, L.V, L.slots, L.dist, L.pred, L.packed);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            const size_t nt = (size_t)L.S * L.n_tails;
            const unsigned tb = (unsigned)std::min<size_t>(std::max<size_t>((nt + 255) / 256, 1), (size_t)sms * 8);
            k_warm_seed<<<tb, 256, 0, st>>>(L);
        } else {
            k_init_fill<<<blocks, 256, 0, st>>>(L.packed, n_packed, L.bitmap, n_words, L.dirty, n_dirty);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_seed<<<(L.S + 127) / 128, 128, 0, st>>>(L);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const size_t smem = relax_smem_bytes(L.tile, L.Q, L.msg_buffer != 0u);
    void* args[] = {const_cast<SolveLaunch*>(&L)};
    if (L.ev_begin && (e = cudaEventRecord(L.ev_begin, st)) != cudaSuccess) return e;
    {
        const bool pr = L.prune_on != 0u, held = L.msg_buffer != 0u, hubs = L.hub_count != 0u;
        const void* k = L.wtype == SSSP_W_F32 ? solve_kernel<WF32>(pr, held, hubs) : solve_kernel<WU32>(pr, held, hubs);
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        if ((e = cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(L.threads), args, smem, st)) != cudaSuccess) return e;
    }
    if (L.ev_end && (e = cudaEventRecord(L.ev_end, st)) != cudaSuccess) return e;
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const unsigned blocks = (unsigned)std::min<size_t>(std::max<size_t>((n_packed + 255) / 256, 1), (size_t)sms * 8);
        if (L.wtype == SSSP_W_F32)
            k_unpack<WF32><<<blocks, 256, 0, st>>>(L.packed, n_packed, L.V, L.slots, L.dist, L.pred);
        else
            k_unpack<WU32><<<blocks, 256, 0, st>>>(L.packed, n_packed, L.V, L.slots, L.dist, L.pred);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the Trishla chunks the idle blocks did not reach
    if (L.prune_on) return trishla_launch(L.prune, L.wtype, &L.hdr->work_next, st);
    return cudaSuccess;
}

uint32_t batched_bitmaps() { return BK_SLOTS; }

cudaError_t batched_max_blocks_per_sm(int wtype, uint32_t threads, uint32_t tile, int* out) {
    const size_t smem = relax_smem_bytes(tile, 0, false);
    cudaError_t e;
    if (wtype == SSSP_W_F32) {
        if ((e = set_smem(k_batched<WF32>, smem)) != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_batched<WF32>, (int)threads, smem);
    }
    if ((e = set_smem(k_batched<WU32>, smem)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_batched<WU32>, (int)threads, smem);
}

cudaError_t launch_batched(const BatchLaunch& L, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(L.hdr, 0, WS_HEADER_BYTES, st)) != cudaSuccess) return e;
    // the dynamic shared-memory limit was raised by batched_max_blocks_per_sm (not a stream
    // operation, so it stays outside any graph capture)
    const size_t smem = relax_smem_bytes(L.tile, 0, false);
    if (L.ev_begin && (e = cudaEventRecord(L.ev_begin, st)) != cudaSuccess) return e;
    if (L.wtype == SSSP_W_F32)
        k_batched<WF32><<<L.grid, L.threads, smem, st>>>(L);
    else
        k_batched<WU32><<<L.grid, L.threads, smem, st>>>(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (L.ev_end && (e = cudaEventRecord(L.ev_end, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace sssp
