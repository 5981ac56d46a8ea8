// fp64.cuh -- FP64 accumulation helpers for the row norms, the residual
// refresh and the final check.
//
// This GPU issues FP64 arithmetic at about 1/64 of its FP32 rate, and an
// FP32 -> FP64 conversion occupies the same pipe as an FP64 FMA.  So an FP32
// value is widened with integer operations (the IEEE 754 binary32 fields
// moved into binary64 position: exact, like the conversion), a warp sums
// several rows at once so that the cross-lane reduction costs one
// transposed butterfly per group of rows instead of one butterfly per row,
// and the next columns' loads are issued before the current ones are used.
#pragma once

#include <cstdint>

#include "reduce.cuh"

namespace csk {

// Exact binary32 -> binary64 with integer operations only.  The sign moves
// to bit 63 and the 23-bit fraction to the top of the 52-bit one; a normal
// number's biased exponent goes from bias 127 to bias 1023 (e + 896); a
// subnormal m * 2^-149 is normalised (its leading one shifted up to the
// implicit bit, the exponent lowered by the shift); +-0 stays +-0; infinities
// and NaNs take exponent 2047 with the fraction (NaN payload) kept.
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    uint32_t ex = e + 896u, fr = m;
    if (e == 0u) {
        const uint32_t sh = (uint32_t)__clz((int)m) - 8u;   // 1..23 for m != 0
        fr = (m << sh) & 0x7FFFFFu;
        ex = m != 0u ? 897u - sh : 0u;
    } else if (e == 255u) {
        ex = 2047u;
    }
    return __hiloint2double((int)(sign | (ex << 20) | (fr >> 3)), (int)(fr << 29));
}
__device__ __forceinline__ double widen(double f) { return f; }

// Loads columns c0, c0 + 32, ..., c0 + 32 (kDotCols - 1) of NR rows (row u
// at a + u * lda, present for u < nrows); absent entries read as 0.
constexpr int kDotCols = 4;

template <int NR, typename TA>
__device__ __forceinline__ void load_cols(TA (&v)[NR][kDotCols], const TA* __restrict__ a, int64_t lda,
                                          int nrows, int c0, int n) {
#pragma unroll
    for (int u = 0; u < NR; ++u)
#pragma unroll
        for (int t = 0; t < kDotCols; ++t) {
            const int c = c0 + 32 * t;
            v[u][t] = (u < nrows && c < n) ? a[(int64_t)u * lda + c] : TA(0);
        }
}

// FP64 dot products of NR rows with x (NR = 1, 2, 4 or 8): row u starts at
// a + u * lda and is present for u < nrows (absent rows sum to 0).  Each lane
// accumulates its columns lane, lane + 32, ... in increasing order with FMA,
// kDotCols of them per row at a time with the next kDotCols already loading
// (double-buffered registers), and the NR partials are combined by
// transpose_sum -- bit for bit the per-row butterfly warp_sum.  Lane l
// returns the sum of row transpose_row<NR>(l).
template <int NR, typename TA, typename TX>
__device__ __forceinline__ double warp_rows_dot_f64(const TA* __restrict__ a, int64_t lda, int nrows,
                                                    const TX* __restrict__ x, int n, int lane) {
    double acc[NR];
#pragma unroll
    for (int u = 0; u < NR; ++u) acc[u] = 0.0;
    TA v[NR][kDotCols], w[NR][kDotCols];
    load_cols<NR>(v, a, lda, nrows, lane, n);
    for (int c0 = lane; c0 < n; c0 += 32 * kDotCols) {
        load_cols<NR>(w, a, lda, nrows, c0 + 32 * kDotCols, n);
#pragma unroll
        for (int t = 0; t < kDotCols; ++t) {
            const int c = c0 + 32 * t;
            if (c < n) {
                const double xv = widen(x[c]);
#pragma unroll
                for (int u = 0; u < NR; ++u) acc[u] = fma(widen(v[u][t]), xv, acc[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < NR; ++u)
#pragma unroll
            for (int t = 0; t < kDotCols; ++t) v[u][t] = w[u][t];
    }
    return transpose_sum<double, NR>(acc, lane);
}

// FP64 sum of squares of NR rows, in the same layout and order.
template <int NR, typename TA>
__device__ __forceinline__ double warp_rows_sq_f64(const TA* __restrict__ a, int64_t lda, int nrows,
                                                   int n, int lane) {
    double acc[NR];
#pragma unroll
    for (int u = 0; u < NR; ++u) acc[u] = 0.0;
    TA v[NR][kDotCols], w[NR][kDotCols];
    load_cols<NR>(v, a, lda, nrows, lane, n);
    for (int c0 = lane; c0 < n; c0 += 32 * kDotCols) {
        load_cols<NR>(w, a, lda, nrows, c0 + 32 * kDotCols, n);
#pragma unroll
        for (int t = 0; t < kDotCols; ++t)
            if (c0 + 32 * t < n)
#pragma unroll
                for (int u = 0; u < NR; ++u) {
                    const double e = widen(v[u][t]);
                    acc[u] = fma(e, e, acc[u]);
                }
#pragma unroll
        for (int u = 0; u < NR; ++u)
#pragma unroll
            for (int t = 0; t < kDotCols; ++t) v[u][t] = w[u][t];
    }
    return transpose_sum<double, NR>(acc, lane);
}

}  // namespace csk
