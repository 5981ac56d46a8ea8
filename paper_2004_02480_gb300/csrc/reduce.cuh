// reduce.cuh -- the argmax candidate of Algorithm 1's selection step and its
// warp / CTA reductions, shared by the loop kernels.
#pragma once

#include <climits>
#include <cstdint>

#include "common.cuh"

namespace csk {

// ----------------------------------------------------- candidate algebra
// Larger key wins; equal keys -> smaller row (first maximiser); NaN keys win
// so that a numerical failure reaches the common decision.
template <typename T>
__device__ __forceinline__ bool better(T ka, int32_t ia, T kb, int32_t ib) {
    const bool na = ka != ka, nb = kb != kb;
    if (na != nb) return na;
    if (na) return ia < ib;
    return ka > kb || (ka == kb && ia < ib);
}

template <typename T>
struct Red {
    T key, alpha, stat;
    int32_t idx;
};

template <typename T>
__device__ __forceinline__ void warp_reduce(Red<T>& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T k2 = __shfl_xor_sync(0xffffffffu, c.key, o);
        const T a2 = __shfl_xor_sync(0xffffffffu, c.alpha, o);
        const int32_t i2 = __shfl_xor_sync(0xffffffffu, c.idx, o);
        c.stat += __shfl_xor_sync(0xffffffffu, c.stat, o);
        if (better(k2, i2, c.key, c.idx)) { c.key = k2; c.alpha = a2; c.idx = i2; }
    }
}

// Warp argmax of FP32 candidates with the integer reduction unit: the key is
// mapped to a monotone 32-bit code (NaN highest, "no candidate" lowest), the
// maximal code and then the smallest row among its holders are found with
// redux.sync, and the winner's step length is fetched from its lane.  Same
// ordering as better(); the statistic is summed with a shuffle tree.
__device__ __forceinline__ void warp_reduce(Red<float>& c) {
    const uint32_t code = c.key != c.key ? 0xFFFFFFFFu
                                         : (c.key < 0.0f ? 0u : __float_as_uint(c.key) + 1u);
    const uint32_t best = __reduce_max_sync(0xffffffffu, code);
    const uint32_t row = __reduce_min_sync(0xffffffffu, code == best ? (uint32_t)c.idx : 0xFFFFFFFFu);
    const unsigned win = __ballot_sync(0xffffffffu, code == best && (uint32_t)c.idx == row);
    const int wl = __ffs(win) - 1;
    c.key = __shfl_sync(0xffffffffu, c.key, wl);
    c.alpha = __shfl_sync(0xffffffffu, c.alpha, wl);
    c.idx = (int32_t)row;
    c.stat = warp_sum(c.stat);
}

// FP64 warp argmax with integer comparisons: non-negative doubles order as
// their bit patterns, so the key becomes a monotone 64-bit code (NaN highest,
// "no candidate" lowest) compared on the integer pipe -- this GPU runs FP64
// at 1/64 of the FP32 rate.  Same ordering as better(); the statistic is
// summed with the same shuffle tree as before.
__device__ __forceinline__ void warp_reduce(Red<double>& c) {
    uint64_t code = c.key != c.key ? ~0ull
                                   : (c.key < 0.0 ? 0ull : (uint64_t)__double_as_longlong(c.key) + 1ull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t c2 = __shfl_xor_sync(0xffffffffu, code, o);
        const double a2 = __shfl_xor_sync(0xffffffffu, c.alpha, o);
        const int32_t i2 = __shfl_xor_sync(0xffffffffu, c.idx, o);
        c.stat += __shfl_xor_sync(0xffffffffu, c.stat, o);
        if (c2 > code || (c2 == code && i2 < c.idx)) { code = c2; c.alpha = a2; c.idx = i2; }
    }
    c.key = code == ~0ull ? (double)NAN
          : code == 0ull ? -1.0 : __longlong_as_double((long long)(code - 1ull));
}

// CTA-wide reduction with a single barrier: warps post their partial results
// in one of two shared buffers (alternating between calls), then every warp
// reduces the posted partials itself, so all threads end with the same bits.
template <typename T, int W = 8>
struct RedShared {
    Red<T> buf[2][W];          // W >= warps per CTA
};

template <typename T, int W>
__device__ __forceinline__ Red<T> block_reduce(Red<T> c, RedShared<T, W>& sh, int& par) {
    warp_reduce(c);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh.buf[par][warp] = c;
    __syncthreads();
    Red<T> r;
    if (lane < (int)(blockDim.x >> 5)) r = sh.buf[par][lane];
    else { r.key = T(-1); r.alpha = T(0); r.stat = T(0); r.idx = INT_MAX; }
    par ^= 1;
    warp_reduce(r);
    return r;
}

// The same, for partials whose candidate is already uniform across each warp
// (Phase A: every lane of a warp holds the row results of that warp), so only
// the statistic needs a warp sum before the cross-warp step.
template <typename T, int W>
__device__ __forceinline__ Red<T> block_reduce_wu(Red<T> c, RedShared<T, W>& sh, int& par) {
    c.stat = warp_sum(c.stat);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh.buf[par][warp] = c;
    __syncthreads();
    Red<T> r;
    if (lane < (int)(blockDim.x >> 5)) r = sh.buf[par][lane];
    else { r.key = T(-1); r.alpha = T(0); r.stat = T(0); r.idx = INT_MAX; }
    par ^= 1;
    warp_reduce(r);
    return r;
}

}  // namespace csk
