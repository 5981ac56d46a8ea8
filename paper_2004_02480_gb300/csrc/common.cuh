// common.cuh -- device helpers shared by the CSK kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "csk.h"

namespace csk {

constexpr int kWarp = 32;

// ---------------------------------------------------------------- hashing
// Count sketch randomness (Definition 1): SplitMix64 output number i+1 of the
// stream seeded with `seed`, used as a counter-based hash of the row index.
__host__ __device__ __forceinline__ uint64_t row_hash(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// h(i): multiply-shift reduction of the high 32 bits onto [0, d).
__host__ __device__ __forceinline__ int32_t row_bucket(uint64_t u, uint32_t d) {
    return (int32_t)(((u >> 32) * (uint64_t)d) >> 32);
}
// D_ii = -1 when bit 0 is set.
__host__ __device__ __forceinline__ bool row_negative(uint64_t u) { return (u & 1ull) != 0; }

// ------------------------------------------------------- memory ordering
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream serialization attribute may be scheduled while its predecessor in
// the stream still runs: pdl_wait() returns once that predecessor has
// completed and its writes are visible (so every read of its output, and
// every write, comes after it); pdl_trigger() lets this kernel's own
// successor be scheduled.  Both do nothing in a kernel launched without the
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Unit of the exchange mailboxes (32 bytes): an FP32 round stores four
// stamped 64-bit words per slot, an FP64 round eight (two units).
struct __align__(32) Slot {
    uint64_t w[4];
};

// Status written into csk_info by the first CTA that fails.
// Threshold of the Section 3 stopping rule (RES <= tol, i.e. stat <= tol *
// norm) for a statistic that is a sum of `terms` non-negative terms, each a
// square of a difference, all rounded in type T: tol * norm shrunk by that
// sum's rounding bound ((terms - 1) u for the additions, 3 u per term, with
// room for the rounding of the threshold itself), so a computed statistic
// at or below it proves the exact one is at most tol * norm.
template <typename T>
__host__ __device__ __forceinline__ T stop_threshold(double tol, double norm, int64_t terms) {
    const double u = sizeof(T) == 4 ? 5.9604644775390625e-8 : 1.1102230246251565e-16;   // 2^-24, 2^-53
    const double f = 1.0 - (double)(terms + 8) * u;      // >= 0: the bound needs (terms + 8) u < 1
    return (T)(tol * norm * (f > 0.0 ? f : 0.0));
}

__device__ __forceinline__ void set_status_once(csk_info* info, int32_t st) {
    atomicCAS(reinterpret_cast<int*>(&info->status), 0, st);
}

}  // namespace csk

#define CSK_CUDA_TRY(expr)                                 \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return CSK_ECUDA;           \
    } while (0)
