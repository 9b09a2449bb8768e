// Shared device helpers and host-side error plumbing of libfbpt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fbpt.h"

namespace fbpt {

// ---- host error handling ---------------------------------------------------------

// Thread-local message behind fbpt_last_error().
void set_error(const std::string& msg);
const char* last_error();

struct Status {
    int code = FBPT_OK;
};

#define FBPT_CUDA_TRY(expr)                                                                        \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            ::fbpt::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                 \
            return _e == cudaErrorMemoryAllocation ? FBPT_ENOMEM : FBPT_ECUDA;                     \
        }                                                                                          \
    } while (0)

#define FBPT_TRY(expr)                 \
    do {                               \
        int _s = (expr);               \
        if (_s != FBPT_OK) return _s;  \
    } while (0)

inline int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int device_sm_count();

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------------------------
//
// Ten rounds of the Philox S-box: the two 32x32 -> 64 products of counter
// words 0 and 2 with the round multipliers, their halves permuted and XORed
// with counter words 1 and 3 and the round key; the key advances by the Weyl
// constants between rounds.

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// The ten round keys of a seed (key advanced by the Weyl constants), computed
// once and reused by every draw of a run.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = a;
        K.k1[r] = b;
        a += kPhiloxW0;
        b += kPhiloxW1;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys& K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[r],
                       (uint32_t)p0);
    }
    return c;
}

// Draws for the four edges 4q .. 4q+3 of sample s (word e & 3 belongs to edge e).
__device__ __forceinline__ uint4 edge_draws4(uint64_t seed, uint64_t s, uint64_t q) {
    return philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(s >> 32), (uint32_t)q, (uint32_t)(q >> 32)),
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Start vertex of sample s: floor(R * n / 2^64), R = 64 bits of the start-domain draw.
__device__ __forceinline__ uint32_t start_vertex(uint64_t seed, uint64_t s, uint32_t n) {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)s, (uint32_t)(s >> 32), 0u, 0x80000000u),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t r = ((uint64_t)o.y << 32) | o.x;
    return (uint32_t)__umul64hi(r, (uint64_t)n);
}

__device__ __forceinline__ bool live(uint32_t draw, uint32_t thr) {
    return thr == 0xFFFFFFFFu || draw < thr;
}

// ---- warp helpers -------------------------------------------------------------------

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Inclusive prefix sum over the 32 lanes (all lanes must call).
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= (uint32_t)d) v += u;
    }
    return v;
}

// Warp-aggregated allocation: each lane asks for `count` slots (0 allowed) of
// the counter; one atomic per warp.  All 32 lanes must call.  Returns this
// lane's first slot.
template <typename T>
__device__ __forceinline__ T warp_alloc(T* ctr, T count) {
    const T incl = warp_incl_scan(count);
    const T total = __shfl_sync(0xffffffffu, incl, 31);
    T base = 0;
    if (lane_id() == 31 && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + incl - count;
}

// Two warp-aggregated allocations at once: lane 31 bumps both counters before
// either result is awaited.  All 32 lanes must call.
template <typename T>
__device__ __forceinline__ void warp_alloc2(T* ca, T na, T& ra, T* cb, T nb, T& rb) {
    const T ia = warp_incl_scan(na), ib = warp_incl_scan(nb);
    const T ta = __shfl_sync(0xffffffffu, ia, 31), tb = __shfl_sync(0xffffffffu, ib, 31);
    T ba = 0, bb = 0;
    if (lane_id() == 31) {
        if (ta) ba = atomicAdd(ca, ta);
        if (tb) bb = atomicAdd(cb, tb);
    }
    ra = __shfl_sync(0xffffffffu, ba, 31) + ia - na;
    rb = __shfl_sync(0xffffffffu, bb, 31) + ib - nb;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

__device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
    uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)v);
    uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
    return ((uint64_t)hi << 32) | lo;
}

}  // namespace fbpt
