// Device-side helpers shared by the libsssp kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sssp.h"

namespace sssp {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t INF32 = 0xFFFFFFFFu;
constexpr unsigned long long INF_KEY = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t F32_INF_BITS = 0x7F800000u;

// Workspace header at the start of every workspace (256 bytes).
struct WsHeader {
    uint32_t status;        // sssp_status of the last call (0 = OK); set with atomicCAS first-error-wins
    uint32_t abort_flag;    // set on a fatal device error so every block stops
    unsigned long long pending;  // queued-but-unprocessed vertices (Sec. III.D counter)
    unsigned long long work_next;  // batched work-queue cursor
    unsigned long long stats[9];   // sssp_stats
    uint32_t pad[(256 - 4 - 4 - 8 - 8 - 72) / 4];
};
static_assert(sizeof(WsHeader) == 256, "header size");

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ double ld_relaxed(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Record the first error of a call; later ones do not overwrite it.
__device__ __forceinline__ void set_status(WsHeader* h, uint32_t st) {
    atomicCAS(&h->status, 0u, st);
}

// Distance arithmetic.  Distances are carried as 32-bit patterns: uint32
// values, or the bits of non-negative float32 values, whose unsigned order is
// the numeric order.  add() returns false when the candidate cannot be
// represented (uint32: >= 0xFFFFFFFF; float32: +inf).
struct WU32 {
    static constexpr int wtype = SSSP_W_U32;
    __device__ __forceinline__ static bool add(uint32_t d, uint32_t w, uint32_t& out) {
        unsigned long long c = (unsigned long long)d + w;
        out = (uint32_t)c;
        return c < 0xFFFFFFFFull;
    }
    __device__ __forceinline__ static bool weight_ok(uint32_t w) { return w >= 1u; }
    __device__ __forceinline__ static uint32_t inf_out() { return INF32; }
    // index of the width-delta distance bucket of d (delta >= 1); non-decreasing in d
    __device__ __forceinline__ static uint32_t bucket(uint32_t d, uint32_t delta) { return d / delta; }
    // end of the fixed bucket [k*delta, (k+1)*delta) that holds d: above d, non-decreasing in d,
    // saturating to 0xFFFFFFFF (every finite distance)
    __device__ __forceinline__ static uint32_t bucket_end(uint32_t d, uint32_t delta) {
        const unsigned long long e = ((unsigned long long)(d / delta) + 1ull) * delta;
        return e < 0xFFFFFFFFull ? (uint32_t)e : 0xFFFFFFFFu;
    }
};

struct WF32 {
    static constexpr int wtype = SSSP_W_F32;
    __device__ __forceinline__ static bool add(uint32_t d, uint32_t w, uint32_t& out) {
        float c = __fadd_rn(__uint_as_float(d), __uint_as_float(w));  // one IEEE rounding, never fused
        out = __float_as_uint(c);
        return out < F32_INF_BITS;
    }
    // positive, finite, not NaN
    __device__ __forceinline__ static bool weight_ok(uint32_t w) { return w > 0u && w < F32_INF_BITS; }
    __device__ __forceinline__ static uint32_t inf_out() { return F32_INF_BITS; }
    // index of the width-delta distance bucket of d: the rounded quotient, truncated (rounding
    // and truncation are both monotone, so the index is non-decreasing in d)
    __device__ __forceinline__ static uint32_t bucket(uint32_t d, uint32_t delta_bits) {
        const float q = __fdiv_rn(__uint_as_float(d), __uint_as_float(delta_bits));
        return q < 4.0e9f ? (uint32_t)q : 4000000000u;
    }
    // end of the fixed bucket that holds d: (floor(d / delta) + 1) * delta, each step rounded
    // once (monotone), and at least one step above d (bit patterns, numeric order)
    __device__ __forceinline__ static uint32_t bucket_end(uint32_t d, uint32_t delta_bits) {
        const float dl = __uint_as_float(delta_bits);
        const float q = floorf(__fdiv_rn(__uint_as_float(d), dl));
        const uint32_t e = __float_as_uint(__fmul_rn(__fadd_rn(q, 1.0f), dl));
        return e > d ? e : d + 1u;
    }
};

}  // namespace sssp
