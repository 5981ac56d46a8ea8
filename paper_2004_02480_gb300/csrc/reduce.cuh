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

// Monotone 64-bit code of an FP64 key, in the order of better(): NaN
// highest, a negative key ("no candidate") lowest, otherwise the bit pattern
// + 1 (non-negative doubles order as their bits).  Integer operations only:
// this GPU runs FP64 -- compares included -- at 1/64 of the FP32 rate.
__device__ __forceinline__ uint64_t key_code(double k) {
    const uint64_t u = (uint64_t)__double_as_longlong(k);
    const uint64_t a = u & 0x7FFFFFFFFFFFFFFFull;
    return a > 0x7FF0000000000000ull ? ~0ull : ((u >> 63) ? 0ull : u + 1ull);
}

// The same order for FP64 keys through their codes.  Keys are r^2 w >= +0,
// NaN, or the negative "no candidate" marker, on which both orders agree.
template <>
__device__ __forceinline__ bool better<double>(double ka, int32_t ia, double kb, int32_t ib) {
    const uint64_t a = key_code(ka), b = key_code(kb);
    return a > b || (a == b && ia < ib);
}

// w < 0 for a row weight (1/||At_j||^2, -1 for a zero row, NaN for a bad
// row); the FP64 form tests the bits (negative and not NaN).
__device__ __forceinline__ bool below_zero(float w) { return w < 0.0f; }
__device__ __forceinline__ bool below_zero(double w) {
    const uint64_t u = (uint64_t)__double_as_longlong(w);
    const uint64_t a = u & 0x7FFFFFFFFFFFFFFFull;
    return (u >> 63) && a != 0ull && a <= 0x7FF0000000000000ull;
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
// at 1/64 of the FP32 rate.  Same ordering as better().  The statistic is
// left alone (see warp_reduce below).
__device__ __forceinline__ void warp_argmax(Red<double>& c) {
    uint64_t code = key_code(c.key);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t c2 = __shfl_xor_sync(0xffffffffu, code, o);
        const double a2 = __shfl_xor_sync(0xffffffffu, c.alpha, o);
        const int32_t i2 = __shfl_xor_sync(0xffffffffu, c.idx, o);
        if (c2 > code || (c2 == code && i2 < c.idx)) { code = c2; c.alpha = a2; c.idx = i2; }
    }
    c.key = code == ~0ull ? (double)NAN
          : code == 0ull ? -1.0 : __longlong_as_double((long long)(code - 1ull));
}

// The FP64 statistic summed by the butterfly, skipped when every lane holds
// +0 (the sum would be +0): FP64 adds occupy the slow pipe, and in most warps
// of a step only a few lanes carry a share of ||x - x*||^2.
__device__ __forceinline__ double warp_sum_nonzero(double v) {
    if (!__any_sync(0xffffffffu, __double_as_longlong(v) != 0)) return v;
    return warp_sum(v);
}

__device__ __forceinline__ void warp_reduce(Red<double>& c) {
    warp_argmax(c);
    c.stat = warp_sum_nonzero(c.stat);
}

// --------------------------------------------------- row sums of a warp
// Sums of a warp's N rows (N = 1, 2, 4, 8, 16; a[u] = this lane's partial of row
// u) by a transposed butterfly: each of the first log2(N) levels halves the
// rows a lane carries, so the N sums cost 5 + N - 1 shuffles and adds instead
// of 5 N, and lane l ends with the sum of row transpose_row<N>(l) (the top
// log2(N) lane bits, bit 4 the row's highest).  Every level adds the same pairs as the xor
// butterfly of warp_sum (16, 8, 4, 2, 1), so each sum is bit for bit the
// warp_sum of its row.
template <int N>
__device__ __forceinline__ int transpose_row(int lane) {
    return N == 16 ? ((lane >> 1) & 15) : N == 8 ? ((lane >> 2) & 7) : N == 4 ? ((lane >> 3) & 3)
         : N == 2 ? ((lane >> 4) & 1) : 0;
}

// The lane of each group holding one row that reports it (lowest free bits 0).
template <int N>
__device__ __forceinline__ bool transpose_rep(int lane) {
    return (lane & (32 / N - 1)) == 0;
}

template <typename T, int N>
__device__ __forceinline__ T transpose_sum(const T (&a)[N], int lane) {
    static_assert(N == 1 || N == 2 || N == 4 || N == 8 || N == 16, "N = 1, 2, 4, 8 or 16");
    T v[N];
#pragma unroll
    for (int u = 0; u < N; ++u) v[u] = a[u];
    int off = 16;
#pragma unroll
    for (int m = N; m > 1; m >>= 1, off >>= 1) {
        const bool hi = lane & off;
#pragma unroll
        for (int i = 0; i < m / 2; ++i) {
            const T send = hi ? v[i] : v[i + m / 2];
            const T keep = hi ? v[i + m / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    T r = v[0];
#pragma unroll
    for (; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    return r;
}

template <int R>
struct Pow2Rows {   // smallest of 1, 2, 4, 8, 16 holding R rows
    static constexpr int N = R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : R <= 8 ? 8 : 16;
};

// CTA-wide reduction with a single barrier: warps post their partial results
// in one of two shared buffers (alternating between calls), then every warp
// reduces the posted partials itself, so all threads end with the same bits.
template <typename T, int W = 8>
struct RedShared {
    Red<T> buf[2][W];          // W >= warps per CTA
    Red<T> res[2];             // FP64: the combined result
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

// FP64: warp 0 alone combines the warps' partials (so the FP64 adds run on
// one warp instead of all of them) and shares the result through shared
// memory, at the price of a second barrier.
template <int W>
__device__ __forceinline__ Red<double> block_reduce(Red<double> c, RedShared<double, W>& sh, int& par) {
    warp_reduce(c);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh.buf[par][warp] = c;
    __syncthreads();
    if (warp == 0) {
        Red<double> r;
        if (lane < (int)(blockDim.x >> 5)) r = sh.buf[par][lane];
        else { r.key = -1.0; r.alpha = 0.0; r.stat = 0.0; r.idx = INT_MAX; }
        warp_reduce(r);
        if (lane == 0) sh.res[par] = r;
    }
    __syncthreads();
    const Red<double> r = sh.res[par];
    par ^= 1;
    return r;
}

// The cross-warp step alone, for a candidate (statistic included) that a
// warp_reduce has already made uniform across each warp.
template <typename T, int W>
__device__ __forceinline__ Red<T> block_combine(const Red<T>& c, RedShared<T, W>& sh, int& par) {
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
