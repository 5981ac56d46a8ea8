// iterate.cu -- the maximal-weighted-residual loop of Algorithm 1 on the
// sketch (At, bt), as one persistent cooperative kernel per solve, plus the
// FP64 final check.
//
// Each CTA owns a contiguous block of rows of At.  A step is
//   Phase A  every CTA scores its rows, key_j = r_j^2 / ||At_j||^2, keeps its
//            best (key, row, alpha = r_j / ||At_j||^2) and a partial of the
//            stopping statistic, and publishes them in its slot;
//   Phase B  every CTA waits for all slots of this round (bounded poll count),
//            reduces them in one fixed order -- so every CTA takes the same
//            decision bit for bit -- tests the stopping rule of Section 3 and
//            applies the projection of Algorithm 1.
// One inter-CTA exchange per step.  Slots alternate between two banks, so a
// fast CTA can never overwrite a slot a slow CTA has still to read.
//
// FP32 solves keep every per-step operation in FP32 (this GPU's FP64 rate is
// a small fraction of its FP32 rate): keys, step lengths and the stopping
// statistic are FP32, and a slot is four 64-bit words that each carry the
// round stamp next to 32 bits of payload, so one relaxed load of each word
// both detects the new round and delivers its data (one L2 round trip).
// FP64 solves use FP64 values throughout (compared and tested through
// integer codes of their bit patterns) and a slot of eight stamped words.
//
// GEMV path: r = bt - At x is recomputed every step (Algorithm 1 as printed).
// Three loops: the CTA's rows of At in registers with x in every warp's
// registers (k_iterate_gemv_reg, FP32), rows and x in shared memory
// (k_iterate_gemv), or rows streamed from global memory through a bulk-copy
// ring every step when they fit neither (k_iterate_gemv_stream: MWRK on A).
// GRAM path: r lives in shared memory, r -= alpha * G[i_k, :] with
// G = At At^T, r_{i_k} = 0 exactly; x is split by columns across CTAs; every
// refresh_every steps r is recomputed as bt - At x with FP64 accumulation.
#include <climits>
#include <cmath>

#include "async.cuh"
#include "common.cuh"
#include "fp64.cuh"
#include "kernels.h"
#include "own_sketch.cuh"
#include "reduce.cuh"

namespace csk {

namespace {

constexpr int kIterThreads = 256;
constexpr int kWarps = kIterThreads / 32;
constexpr int64_t kDefaultSpin = 1ll << 22;
constexpr int kRowsPerWarp = 8;          // rows a warp scores in one pass at most (1, 2, 4 or 8)
constexpr int kRefreshRows = 4;          // rows a warp sums at once in the FP64 refresh

// ---------------------------------------------------------- exchanges
// Mailboxes: bank (round parity) x destination CTA x source CTA, 32 bytes
// each.  A CTA writes its candidate into every destination's mailbox and
// polls only its own, so no cache line is polled by more than one CTA.
__device__ __forceinline__ void st_relaxed_v2(uint64_t* p, uint64_t a, uint64_t b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const uint64_t* p, uint64_t& a, uint64_t& b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ Slot* mailbox(Slot* slots, uint32_t round, int dest, int src, int G) {
    return slots + ((size_t)(round & 1u) * G + dest) * G + src;
}

// Rows the chosen candidate's data will be read from after an exchange: the
// bytes [base + idx * ld, + bytes) of row idx < rows.  Each polling warp
// prefetches them into L1 for its own best candidate, before the CTA-wide
// reduction picks the winner among the warps' bests (the winner is always one
// of them), so the read after the exchange finds them on chip.
struct RowPrefetch {
    const char* base = nullptr;
    int64_t ld = 0;            // bytes between rows
    int bytes = 0;             // <= 32 lines of 128 bytes
    int rows = 0;
};

__device__ __forceinline__ void prefetch_row(const RowPrefetch& pf, int32_t idx) {
    if (!pf.base || (uint32_t)idx >= (uint32_t)pf.rows) return;
    const uintptr_t r = reinterpret_cast<uintptr_t>(pf.base) + (uintptr_t)idx * (uintptr_t)pf.ld;
    const uintptr_t a = (r & ~(uintptr_t)127) + 128u * (threadIdx.x & 31);
    if (a < r + (uintptr_t)pf.bytes) asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}

// FP32: four stamped words per slot.
// With `acquire`, every polling thread fences after seeing the new round, so
// plain data the other CTAs stored before publishing is visible afterwards.
// Among G participants, this CTA being participant b (by default the whole
// grid, CTA b = blockIdx.x).
__device__ __forceinline__ bool exchange(Slot* slots, uint32_t round, Red<float>& c,
                                         int64_t spin_limit, int fault_inject, csk_info* info,
                                         RedShared<float>& sh, int& par, bool acquire = false,
                                         const RowPrefetch& pf = RowPrefetch(), int G = 0,
                                         int b = -1) {
    if (G == 0) { G = gridDim.x; b = blockIdx.x; }
    const uint64_t stamp = (uint64_t)(round + 1u) << 32;
    if (!(fault_inject && b == 0))
        for (int t = threadIdx.x; t < G; t += blockDim.x) {
            uint64_t* w = reinterpret_cast<uint64_t*>(mailbox(slots, round, t, b, G));
            st_relaxed_v2(w, stamp | __float_as_uint(c.key), stamp | __float_as_uint(c.alpha));
            st_relaxed_v2(w + 2, stamp | __float_as_uint(c.stat), stamp | (uint32_t)c.idx);
        }
    Red<float> g;
    g.key = -1.0f; g.alpha = 0.0f; g.stat = 0.0f; g.idx = INT_MAX;
    int timed_out = 0;
    for (int t = threadIdx.x; t < G; t += blockDim.x) {
        const uint64_t* w = reinterpret_cast<const uint64_t*>(mailbox(slots, round, b, t, G));
        uint64_t v0, v1, v2, v3;
        int64_t spins = 0;
        for (;;) {
            ld_relaxed_v2(w, v0, v1);
            ld_relaxed_v2(w + 2, v2, v3);
            const uint64_t hi = stamp >> 32;
            if ((v0 >> 32) == hi && (v1 >> 32) == hi && (v2 >> 32) == hi && (v3 >> 32) == hi) break;
            if (++spins > spin_limit) { timed_out = 1; break; }
        }
        if (timed_out) break;
        if (acquire) __threadfence();
        const float k2 = __uint_as_float((uint32_t)v0);
        const int32_t i2 = (int32_t)(uint32_t)v3;
        g.stat += __uint_as_float((uint32_t)v2);
        if (better(k2, i2, g.key, g.idx)) { g.key = k2; g.alpha = __uint_as_float((uint32_t)v1); g.idx = i2; }
    }
    if (__syncthreads_or(timed_out)) {
        if (threadIdx.x == 0) set_status_once(info, CSK_ETIMEOUT);
        return false;
    }
    if (pf.base) {
        warp_reduce(g);
        prefetch_row(pf, g.idx);
        c = block_combine(g, sh, par);
    } else {
        c = block_reduce(g, sh, par);
    }
    return true;
}

// FP64: a slot is eight 64-bit words (64 bytes), each carrying the round
// stamp in its high half beside 32 payload bits: key, step length and
// statistic as two halves each, then the row.  As for FP32, one relaxed load
// of each word both detects the new round and delivers the data, and a
// reader that sees the stamp on all eight words has a consistent payload.
__device__ __forceinline__ uint64_t* mailbox64(Slot* slots, uint32_t round, int dest, int src) {
    const int G = gridDim.x;
    return reinterpret_cast<uint64_t*>(slots) + ((((size_t)(round & 1u) * G + dest) * G + src) << 3);
}

__device__ __forceinline__ bool exchange(Slot* slots, uint32_t round, Red<double>& c,
                                         int64_t spin_limit, int fault_inject, csk_info* info,
                                         RedShared<double>& sh, int& par) {
    const int G = gridDim.x, b = blockIdx.x;
    const uint64_t stamp = (uint64_t)(round + 1u) << 32;
    if (!(fault_inject && b == 0)) {
        const uint64_t kb = (uint64_t)__double_as_longlong(c.key);
        const uint64_t ab = (uint64_t)__double_as_longlong(c.alpha);
        const uint64_t sb = (uint64_t)__double_as_longlong(c.stat);
        for (int t = threadIdx.x; t < G; t += blockDim.x) {
            uint64_t* w = mailbox64(slots, round, t, b);
            st_relaxed_v2(w, stamp | (kb >> 32), stamp | (kb & 0xFFFFFFFFull));
            st_relaxed_v2(w + 2, stamp | (ab >> 32), stamp | (ab & 0xFFFFFFFFull));
            st_relaxed_v2(w + 4, stamp | (sb >> 32), stamp | (sb & 0xFFFFFFFFull));
            st_relaxed_v2(w + 6, stamp | (uint32_t)c.idx, stamp);
        }
    }
    Red<double> g;
    g.key = -1.0; g.alpha = 0.0; g.stat = 0.0; g.idx = INT_MAX;
    int timed_out = 0;
    const uint64_t hi = stamp >> 32;
    for (int t = threadIdx.x; t < G; t += blockDim.x) {
        const uint64_t* w = mailbox64(slots, round, b, t);
        uint64_t v[8];
        int64_t spins = 0;
        for (;;) {
            ld_relaxed_v2(w, v[0], v[1]);
            ld_relaxed_v2(w + 2, v[2], v[3]);
            ld_relaxed_v2(w + 4, v[4], v[5]);
            ld_relaxed_v2(w + 6, v[6], v[7]);
            bool all = true;
#pragma unroll
            for (int q = 0; q < 8; ++q) all &= (v[q] >> 32) == hi;
            if (all) break;
            if (++spins > spin_limit) { timed_out = 1; break; }
        }
        if (timed_out) break;
        const double k2 = __longlong_as_double((long long)((v[0] << 32) | (v[1] & 0xFFFFFFFFull)));
        const double a2 = __longlong_as_double((long long)((v[2] << 32) | (v[3] & 0xFFFFFFFFull)));
        const double s2 = __longlong_as_double((long long)((v[4] << 32) | (v[5] & 0xFFFFFFFFull)));
        const int32_t i2 = (int32_t)(uint32_t)v[6];
        g.stat += s2;
        if (better(k2, i2, g.key, g.idx)) { g.key = k2; g.alpha = a2; g.idx = i2; }
    }
    if (__syncthreads_or(timed_out)) {
        if (threadIdx.x == 0) set_status_once(info, CSK_ETIMEOUT);
        return false;
    }
    c = block_reduce(g, sh, par);
    return true;
}

// Decision shared by every CTA after an exchange (Section 3 stopping rule,
// tested before the step).  Returns a csk_status to stop with, or INT_MIN to
// continue.
template <typename T>
__device__ __forceinline__ int decide(T stat, T threshold, int64_t k, int64_t max_iter, T key) {
    if (stat <= threshold) return CSK_OK;
    if (k >= max_iter) return CSK_MAXITER;
    if (key != key || key < T(0)) return CSK_ENUMERIC;   // NaN, or no non-zero row
    if (key == T(0)) return CSK_OK;                      // every residual is exactly 0
    return INT_MIN;
}

// FP64: the same tests on the integer pipe.  stat is a sum of squares and
// threshold = tol * ||.||^2 with tol >= 0, so both are +0, positive, Inf or
// NaN, and for those "stat <= threshold" is an unsigned comparison of the bit
// patterns unless one of them is NaN.  The key tests read its code.
template <>
__device__ __forceinline__ int decide<double>(double stat, double threshold, int64_t k,
                                              int64_t max_iter, double key) {
    const uint64_t sb = (uint64_t)__double_as_longlong(stat);
    const uint64_t tb = (uint64_t)__double_as_longlong(threshold);
    const uint64_t kInf = 0x7FF0000000000000ull;
    if ((sb & ~(1ull << 63)) <= kInf && (tb & ~(1ull << 63)) <= kInf &&
        ((sb << 1) == 0 || sb <= tb))
        return CSK_OK;
    if (k >= max_iter) return CSK_MAXITER;
    const uint64_t kc = key_code(key);
    if (kc == ~0ull || kc == 0ull) return CSK_ENUMERIC;     // NaN, or no non-zero row
    if (kc == 1ull) return CSK_OK;                           // every residual is exactly 0
    return INT_MIN;
}

__device__ __forceinline__ void finish(csk_info* info, int status, int64_t k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info->iters = k;
        if (status != CSK_OK) set_status_once(info, status);
    }
}

template <typename T>
__device__ __forceinline__ T weight_of(double N) {
    // 1/||At_j||^2; -1 marks a zero row (excluded from the argmax); NaN (a
    // NaN/Inf row) is kept so that the failure reaches the decision
    return N > 0.0 ? (T)(1.0 / N) : (N == 0.0 ? T(-1) : (T)NAN);
}

// This lane's FP64 partial of a . x over columns lane, lane + 32, ... (in that
// order), with sixteen loads of `a` in flight at a time.
template <typename TA, typename TX>
__device__ __forceinline__ double lane_dot_f64(const TA* __restrict__ a, const TX* __restrict__ x,
                                               int n, int lane) {
    double acc = 0.0;
    for (int c0 = lane; c0 < n; c0 += 32 * 16) {
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int c = c0 + 32 * u;
            v[u] = c < n ? (double)a[c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int c = c0 + 32 * u;
            if (c < n) acc = fma(v[u], (double)x[c], acc);
        }
    }
    return acc;
}

// Sum of squares of a 16-byte chunk of x - x*, rounded in a fixed order (no
// contraction left to the compiler), so the register and streamed loops
// compute the stopping statistic identically.
__device__ __forceinline__ float chunk_sq(const float (&t)[4]) {
    float s = __fmul_rn(t[0], t[0]);
    s = __fmaf_rn(t[1], t[1], s);
    s = __fmaf_rn(t[2], t[2], s);
    return __fmaf_rn(t[3], t[3], s);
}
__device__ __forceinline__ double chunk_sq(const double (&t)[2]) {
    return __fma_rn(t[1], t[1], __dmul_rn(t[0], t[0]));
}

// ------------------------------------------------------------ GEMV path
// Shared memory: x (npad) | w2 (Rpad) | bt (Rpad) | x* slice (spad) | At rows
// Loads of rows of At from other CTAs: through the read-only path, except in
// the fused kernels, where At is written earlier in the same launch (then
// coherent L2 loads).
template <bool FUSED, typename V>
__device__ __forceinline__ V ld_row(const V* q) {
    if (FUSED) return __ldcg(q);
    return __ldg(q);
}

// The loop body; stop_norm is ||x*||^2 (or ||bt||^2 without x*), round0 the
// exchange round it starts at.
template <typename T, int NR, bool FUSED>
__device__ __forceinline__ void gemv_loop(const IterProblem& p, int R, int cache_rows,
                                          double stop_norm, uint32_t round0) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ RedShared<T> sh;
    int par = 0;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int n = p.n, d = p.d;
    const int r0 = min(d, b * R), r1 = min(d, r0 + R), nr = r1 - r0;
    const int c0 = (int)((int64_t)n * b / G), c1 = (int)((int64_t)n * (b + 1) / G);
    const int npad = (n + 3) & ~3, Rpad = (R + 3) & ~3, spad = ((n + G - 1) / G + 4) & ~3;
    // FP64 with x*: every CTA keeps all of x* and computes ||x - x*||^2 itself
    // (one warp, during the exchange's poll), so the FP64 statistic leaves the
    // CTA reductions and the exchange; FP32 sums its share of the columns
    constexpr bool kLocalStat = sizeof(T) == 8;
    T* xs = reinterpret_cast<T*>(dsm);
    T* w2s = xs + npad;
    T* bts = w2s + Rpad;
    T* xss = bts + Rpad;
    T* As = xss + (kLocalStat ? npad : spad);
    __shared__ T stat_local;
    const T* At = static_cast<const T*>(p.At);
    const T* bt = static_cast<const T*>(p.bt);
    const T* x0 = static_cast<const T*>(p.x0);
    const T* xstar = static_cast<const T*>(p.xstar);

    for (int c = tid; c < n; c += blockDim.x) xs[c] = x0 ? x0[c] : T(0);
    for (int q = tid; q < nr; q += blockDim.x) {
        w2s[q] = weight_of<T>(p.N2[r0 + q]);
        bts[q] = bt[r0 + q];
    }
    if (xstar) {
        if (kLocalStat)
            for (int c = tid; c < n; c += blockDim.x) xss[c] = xstar[c];
        else
            for (int c = c0 + tid; c < c1; c += blockDim.x) xss[c - c0] = xstar[c];
    }
    if (cache_rows)
        for (int64_t e = tid; e < (int64_t)nr * n; e += blockDim.x) {
            const int q = (int)(e / n), c = (int)(e - (int64_t)q * n);
            As[e] = At[(int64_t)(r0 + q) * p.ld + c];
        }
    __syncthreads();
    // RES <= tol  <=>  stat <= tol ||x*||^2 (sum over the n columns, or the d rows without x*)
    const T threshold = stop_threshold<T>(p.tol, stop_norm, p.xstar ? p.n : p.d);
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    const int64_t lda = cache_rows ? (int64_t)n : p.ld;
    const T* Abase = cache_rows ? As : At + (int64_t)r0 * p.ld;
    // 128-bit row loads: FP32, n % 4 == 0 and 16-byte aligned rows
    const bool vec4 = sizeof(T) == 4 && (n & 3) == 0 && (lda & 3) == 0 &&
                      (reinterpret_cast<uintptr_t>(Abase) & 15) == 0;
    uint32_t round = round0;
    int64_t k = 0;
    int status = CSK_OK;
    for (;;) {
        // Phase A: residuals of the owned rows.  FP32: warp w scores rows
        // w, w + kWarps, ... (round robin), up to NR in one pass over the
        // columns so their loads overlap.  FP64: warp w scores NR
        // consecutive rows w NR, ..., then w NR + kWarps NR, ...: this GPU
        // issues an FP64 warp instruction at the same cost whatever its
        // active lanes, so few warps with many rows each (one transposed
        // butterfly and one key computation for NR rows) take fewer FP64
        // instructions than many warps with few rows.
        constexpr bool kContig = sizeof(T) == 8;
        Red<T> c;
        c.key = T(-1); c.alpha = T(0); c.stat = T(0); c.idx = INT_MAX;
        for (int base = kContig ? warp * NR : warp; base < nr; base += kWarps * NR) {
            const int myrows = kContig ? min(NR, nr - base)
                                       : min(NR, (nr - base + kWarps - 1) / kWarps);
            const int rstride = kContig ? 1 : kWarps;      // between a warp's rows of one pass
            T acc[NR];
#pragma unroll
            for (int u = 0; u < NR; ++u) acc[u] = T(0);
            if (vec4) {
                const float4* x4 = reinterpret_cast<const float4*>(xs);
                for (int c4 = lane; c4 < (n >> 2); c4 += 32) {
                    const float4 xv = x4[c4];
#pragma unroll
                    for (int u = 0; u < NR; ++u)
                        if (u < myrows) {
                            const float4 a = reinterpret_cast<const float4*>(
                                Abase + (int64_t)(base + u * rstride) * lda)[c4];
                            acc[u] = fma((T)a.x, (T)xv.x, acc[u]);
                            acc[u] = fma((T)a.y, (T)xv.y, acc[u]);
                            acc[u] = fma((T)a.z, (T)xv.z, acc[u]);
                            acc[u] = fma((T)a.w, (T)xv.w, acc[u]);
                        }
                }
            } else {
                for (int col = lane; col < n; col += 32) {
                    const T xv = xs[col];
#pragma unroll
                    for (int u = 0; u < NR; ++u)
                        if (u < myrows) acc[u] = fma(Abase[(int64_t)(base + u * rstride) * lda + col], xv, acc[u]);
                }
            }
            // lane l ends with row u(l)'s sum, bit for bit the warp_sum of that row
            const T sum = transpose_sum<T, NR>(acc, lane);
            const int u = transpose_row<NR>(lane);
            if (transpose_rep<NR>(lane) && u < myrows) {
                const int q = base + u * rstride;
                const T r = bts[q] - sum;
                const T w = w2s[q];
                if (!below_zero(w)) {
                    const T key = r * r * w;
                    if (better(key, r0 + q, c.key, c.idx)) { c.key = key; c.alpha = r * w; c.idx = r0 + q; }
                }
                if (!xstar) c.stat += r * r;
            }
        }
        if (xstar && !kLocalStat)
            for (int col = c0 + tid; col < c1; col += blockDim.x) {
                const T t = xs[col] - xss[col - c0];
                c.stat += t * t;
            }
        c = block_reduce(c, sh, par);    // candidates differ across lanes
        if (xstar && kLocalStat && warp == kWarps - 1) {
            // the last warp polls no mailbox while the grid has at most
            // 32 (kWarps - 1) CTAs: it sums ||x - x*||^2 (columns lane,
            // lane + 32, ... in order, then the butterfly) meanwhile
            T acc = T(0);
            for (int col = lane; col < n; col += 32) {
                const T t = xs[col] - xss[col];
                acc = fma(t, t, acc);
            }
            acc = warp_sum(acc);
            if (lane == 0) stat_local = acc;
        }
        // Phase B
        if (!exchange(p.slots, round, c, spin, p.fault_inject, p.info, sh, par)) {
            status = CSK_ETIMEOUT;
            break;
        }
        ++round;
        const T stat = (xstar && kLocalStat) ? stat_local : c.stat;
        const int dec = decide(stat, threshold, k, p.max_iter, c.key);
        if (dec != INT_MIN) { status = dec; break; }
        if (b == 0 && tid == 0 && p.ik_log && k < p.ik_log_len) p.ik_log[k] = c.idx;
        if (b == 0 && p.x_log && k < p.x_log_len)
            for (int col = tid; col < n; col += blockDim.x) static_cast<T*>(p.x_log)[k * n + col] = xs[col];
        // projection onto row i_k: x += alpha * At_{i_k}^T (same in every CTA)
        const T* arow = At + (int64_t)c.idx * p.ld;
        for (int col = tid; col < n; col += blockDim.x) xs[col] = fma(c.alpha, ld_row<FUSED>(arow + col), xs[col]);
        __syncthreads();
        ++k;
    }
    if (b == 0) {
        T* xo = static_cast<T*>(p.x_out);
        for (int col = tid; col < n; col += blockDim.x) xo[col] = xs[col];
    }
    finish(p.info, status, k);
}

template <typename T, int NR>
__global__ void __launch_bounds__(kIterThreads, 1)
k_iterate_gemv(IterProblem p, int R, int cache_rows) {
    gemv_loop<T, NR, false>(p, R, cache_rows, *p.stop_norm, 0);
}

// ------------------------------------------------ GEMV path, registers
// FP32 variant for n <= 128 * CPL (n % 4 == 0) and at most kWarps * RPW rows
// per CTA: warp w keeps rows w, w + kWarps, ... of At in registers (lane l
// holds the float4 columns l, l + 32, ...), and every warp keeps x for the
// same columns in registers, so a step touches no shared memory except the
// CTA reduction.  The projection is applied by every warp to its own copy
// of x (identical arithmetic everywhere); float4 column c4 of the
// ||x - x*||^2 statistic is counted by CTA c4 % grid alone.
template <int RPW, int CPL, bool FUSED>
__device__ __forceinline__ void reg_loop(const IterProblem& p, int R, double stop_norm,
                                         uint32_t round0) {
    __shared__ RedShared<float> sh;
    __shared__ float stat_local;
    int par = 0;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int n = p.n, d = p.d, n4 = n >> 2;
    const int r0 = min(d, b * R), r1 = min(d, r0 + R), nr = r1 - r0;
    const float* At = static_cast<const float*>(p.At);
    const float* bt = static_cast<const float*>(p.bt);
    const float* x0 = static_cast<const float*>(p.x0);
    const float* xstar = static_cast<const float*>(p.xstar);
    const bool stat_owner = (b == 0 && warp == 0);

    float4 a[RPW][CPL];
    float btu[RPW], wu[RPW];
    bool has[RPW];
#pragma unroll
    for (int u = 0; u < RPW; ++u) {
        const int q = warp + kWarps * u;
        has[u] = q < nr;
        btu[u] = has[u] ? bt[r0 + q] : 0.0f;
        wu[u] = has[u] ? weight_of<float>(p.N2[r0 + q]) : -1.0f;
        const float4* row = reinterpret_cast<const float4*>(At + (int64_t)(r0 + (has[u] ? q : 0)) * p.ld);
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int c4 = lane + 32 * i;
            a[u][i] = (has[u] && c4 < n4) ? row[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    float4 xr[CPL], xsr[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        const int c4 = lane + 32 * i;
        xr[i] = (x0 && c4 < n4) ? reinterpret_cast<const float4*>(x0)[c4] : make_float4(0.f, 0.f, 0.f, 0.f);
        xsr[i] = (xstar && c4 < n4) ? reinterpret_cast<const float4*>(xstar)[c4]
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float threshold = stop_threshold<float>(p.tol, stop_norm, p.xstar ? p.n : p.d);
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    // With x*, the last warp (which polls no mailbox: the grid has at most
    // 32 (kWarps - 1) CTAs) sums ||x - x*||^2 over all columns from its own
    // copy of x during the exchange, so every CTA holds the same statistic
    // and it stays out of the candidates and the exchange
    const bool local_stat = xstar != nullptr && (int)gridDim.x <= 32 * (kWarps - 1);
    uint32_t round = round0;
    int64_t k = 0;
    int status = CSK_OK;
    for (;;) {
        float dot[RPW];
#pragma unroll
        for (int u = 0; u < RPW; ++u) {
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                acc = fmaf(a[u][i].x, xr[i].x, acc);
                acc = fmaf(a[u][i].y, xr[i].y, acc);
                acc = fmaf(a[u][i].z, xr[i].z, acc);
                acc = fmaf(a[u][i].w, xr[i].w, acc);
            }
            dot[u] = acc;
        }
        // each lane ends with one row's residual and scores it; the CTA
        // reduction picks the best of all lanes
        constexpr int N = Pow2Rows<RPW>::N;
        float part[N];
#pragma unroll
        for (int u = 0; u < N; ++u) part[u] = u < RPW ? dot[u] : 0.0f;
        const float sum = transpose_sum<float, N>(part, lane);
        const int u = transpose_row<N>(lane);
        float bt_u = 0.0f, w_u = -1.0f;
        bool has_u = false;
#pragma unroll
        for (int v = 0; v < RPW; ++v)
            if (v == u) { bt_u = btu[v]; w_u = wu[v]; has_u = has[v]; }
        Red<float> c;
        c.key = -1.0f; c.alpha = 0.0f; c.stat = 0.0f; c.idx = INT_MAX;
        if (transpose_rep<N>(lane) && has_u) {
            const float r = bt_u - sum;
            if (!(w_u < 0.0f)) {
                c.key = r * r * w_u;
                c.alpha = r * w_u;
                c.idx = r0 + warp + kWarps * u;
            }
            if (!xstar) c.stat += r * r;
        }
        if (xstar && !local_stat && warp == 0) {
            // float4 column c4 is counted by CTA c4 % G only
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                if (lane + 32 * i < n4 && (lane + 32 * i) % (int)gridDim.x == b) {
                    const float t[4] = {xr[i].x - xsr[i].x, xr[i].y - xsr[i].y,
                                        xr[i].z - xsr[i].z, xr[i].w - xsr[i].w};
                    c.stat += chunk_sq(t);
                }
            }
        }
        c = block_reduce(c, sh, par);    // candidates differ across lanes
        if (local_stat && warp == kWarps - 1) {
            float acc = 0.0f;
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                if (lane + 32 * i < n4) {
                    const float t[4] = {xr[i].x - xsr[i].x, xr[i].y - xsr[i].y,
                                        xr[i].z - xsr[i].z, xr[i].w - xsr[i].w};
                    acc += chunk_sq(t);
                }
            }
            acc = warp_sum(acc);
            if (lane == 0) stat_local = acc;
        }
        if (!exchange(p.slots, round, c, spin, p.fault_inject, p.info, sh, par)) {
            status = CSK_ETIMEOUT;
            break;
        }
        ++round;
        // (stat_local was written before the exchange's barriers)
        const int dec = decide(local_stat ? stat_local : c.stat, threshold, k, p.max_iter, c.key);
        if (dec != INT_MIN) { status = dec; break; }
        if (stat_owner && lane == 0 && p.ik_log && k < p.ik_log_len) p.ik_log[k] = c.idx;
        if (stat_owner && p.x_log && k < p.x_log_len)
#pragma unroll
            for (int i = 0; i < CPL; ++i)
                if (lane + 32 * i < n4)
                    reinterpret_cast<float4*>(static_cast<float*>(p.x_log) + k * n)[lane + 32 * i] = xr[i];
        // projection onto row i_k, applied by every warp to its copy of x
        const float4* arow = reinterpret_cast<const float4*>(At + (int64_t)c.idx * p.ld);
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int c4 = lane + 32 * i;
            if (c4 < n4) {
                const float4 v = ld_row<FUSED>(arow + c4);
                xr[i].x = fmaf(c.alpha, v.x, xr[i].x);
                xr[i].y = fmaf(c.alpha, v.y, xr[i].y);
                xr[i].z = fmaf(c.alpha, v.z, xr[i].z);
                xr[i].w = fmaf(c.alpha, v.w, xr[i].w);
            }
        }
        ++k;
    }
    if (stat_owner) {
        float4* xo = reinterpret_cast<float4*>(p.x_out);
#pragma unroll
        for (int i = 0; i < CPL; ++i)
            if (lane + 32 * i < n4) xo[lane + 32 * i] = xr[i];
    }
    finish(p.info, status, k);
}

template <int RPW, int CPL>
__global__ void __launch_bounds__(kIterThreads, 1)
k_iterate_gemv_reg(IterProblem p, int R) {
    reg_loop<RPW, CPL, false>(p, R, *p.stop_norm, 0);
}

// ------------------------------------------- fused sketch and loop
// One cooperative launch for the whole of Algorithm 1 on a sketch: the CTA
// that will own rows [r0, r1) of At in the loop first forms them itself.
//   1. every CTA stores the 16-bit buckets h(i) of a share of the rows
//      (Definition 1), then one exchange round (acquire) makes them visible;
//   2. the CTA sketches buckets [r0, r1) exactly as csk_sketch's bucket-owner
//      kernel does (own_sketch.cuh: rows in ascending order, the same FP
//      additions), writing At, bt and the FP64 row norms of its rows;
//   3. the stopping norm: ||x*||^2, computed by every CTA in the same order,
//      or ||bt||^2 from the CTAs' FP64 partials after a second exchange round
//      (acquire), which also makes every CTA's rows of At visible to the
//      projections of the loop;
//   4. the loop, from exchange round 2 on, reading other CTAs' rows of At
//      with coherent loads.
// The sort chain, the segmented sums, the norms and the loop thus run in one
// kernel; only the status record's initialisation and the FP64 final check
// are launches of their own.
struct FusedSketch {
    const void* A;
    int64_t lda, m;
    const void* b;
    uint64_t seed;
    uint16_t* h;          // m buckets (scratch)
    int32_t* perm;        // m (scratch)
    int32_t* off;         // d + 1 (scratch)
    double* part;         // one FP64 partial per CTA (scratch)
    int cap;              // rows a CTA lists in shared memory
};

__device__ __forceinline__ double block_sum_f64_fixed(double v, double* sh) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[w];     // the same order in every CTA
    __syncthreads();
    return t;
}

// Steps 1-3 above; false (status set) when an exchange round ran out.
template <typename T, int V, int CPL>
__device__ __forceinline__ bool fused_prologue(const IterProblem& p, const FusedSketch& f, int R,
                                               int32_t* smem_rows, double* stop_out,
                                               uint32_t& round) {
    __shared__ OwnShared osh;
    __shared__ RedShared<float> rsh;
    __shared__ double dsh[32];
    int par = 0;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    hash16_range(f.m, (uint32_t)p.d, f.seed, f.h, (int64_t)b * blockDim.x + tid,
                 (int64_t)G * blockDim.x);
    __threadfence();
    __syncthreads();
    Red<float> z;
    z.key = -1.0f; z.alpha = 0.0f; z.stat = 0.0f; z.idx = INT_MAX;
    if (!exchange(p.slots, round, z, spin, p.fault_inject, p.info, rsh, par, true)) return false;
    ++round;
    const int r0 = min(p.d, b * R), r1 = min(p.d, r0 + R);
    T* At = static_cast<T*>(const_cast<void*>(p.At));
    T* bt = static_cast<T*>(const_cast<void*>(p.bt));
    double* N2 = const_cast<double*>(p.N2);
    own_sketch_cta<T, V, CPL>(static_cast<const T*>(f.A), f.lda, p.n, f.m,
                              static_cast<const T*>(f.b), 1, 1, f.h, p.d, f.seed, f.cap, At, bt,
                              N2, f.perm, f.off, r0, r1, smem_rows, smem_rows + f.cap, osh);
    __syncthreads();
    const T* xstar = static_cast<const T*>(p.xstar);
    double sq = 0.0;
    if (xstar) {
        for (int c = tid; c < p.n; c += blockDim.x) sq += (double)xstar[c] * (double)xstar[c];
    } else {
        for (int q = r0 + tid; q < r1; q += blockDim.x) sq += (double)bt[q] * (double)bt[q];
    }
    sq = block_sum_f64_fixed(sq, dsh);
    if (!xstar && tid == 0) f.part[b] = sq;
    __threadfence();
    __syncthreads();
    z.key = -1.0f; z.alpha = 0.0f; z.stat = 0.0f; z.idx = INT_MAX;
    if (!exchange(p.slots, round, z, spin, p.fault_inject, p.info, rsh, par, true)) return false;
    ++round;
    if (!xstar) {
        sq = 0.0;
        for (int q = 0; q < G; ++q) sq += __ldcg(f.part + q);    // the same order in every CTA
    }
    *stop_out = sq;
    __syncthreads();
    return true;
}

template <typename T, int NR, int V, int CPL>
__global__ void __launch_bounds__(kIterThreads, 1)
k_fused_gemv(IterProblem p, FusedSketch f, int R, int cache_rows) {
    extern __shared__ __align__(128) unsigned char dsm_f[];
    uint32_t round = 0;
    double stop = 0.0;
    if (!fused_prologue<T, V, CPL>(p, f, R, reinterpret_cast<int32_t*>(dsm_f), &stop, round)) {
        finish(p.info, CSK_ETIMEOUT, 0);
        return;
    }
    gemv_loop<T, NR, true>(p, R, cache_rows, stop, round);
}

template <int RPW, int CPL>
__global__ void __launch_bounds__(kIterThreads, 1)
k_fused_reg(IterProblem p, FusedSketch f, int R) {
    extern __shared__ __align__(128) unsigned char dsm_f[];
    uint32_t round = 0;
    double stop = 0.0;
    if (!fused_prologue<float, 4, 4>(p, f, R, reinterpret_cast<int32_t*>(dsm_f), &stop, round)) {
        finish(p.info, CSK_ETIMEOUT, 0);
        return;
    }
    reg_loop<RPW, CPL, true>(p, R, stop, round);
}

// Register-resident variants: (rows per warp, float4 per lane per row); 9 and
// 10 rows a warp (rows of up to 512 columns) let fewer CTAs hold the sketch.
#define CSK_REG_VARIANTS(X) \
    X(1, 1) X(2, 1) X(3, 1) X(4, 1) X(6, 1) X(8, 1) \
    X(1, 2) X(2, 2) X(3, 2) X(4, 2) X(6, 2) X(8, 2) \
    X(1, 4) X(2, 4) X(3, 4) X(4, 4) X(5, 4) X(6, 4) X(7, 4) X(8, 4) X(9, 4) X(10, 4)

// Fused register loops for rows of 257..512 columns (4 float4 per lane).
#define CSK_FUSED_REG_VARIANTS(X) \
    X(1, 4) X(2, 4) X(3, 4) X(4, 4) X(5, 4) X(6, 4) X(7, 4) X(8, 4) X(9, 4) X(10, 4)

const void* fused_reg_kernel(int rpw, int cpl) {
#define CSK_PICK(RPWv, CPLv) \
    if (rpw == RPWv && cpl == CPLv) return (const void*)k_fused_reg<RPWv, CPLv>;
    CSK_FUSED_REG_VARIANTS(CSK_PICK)
#undef CSK_PICK
    return nullptr;
}

const void* reg_kernel(int rpw, int cpl) {
#define CSK_PICK(RPWv, CPLv) \
    if (rpw == RPWv && cpl == CPLv) return (const void*)k_iterate_gemv_reg<RPWv, CPLv>;
    CSK_REG_VARIANTS(CSK_PICK)
#undef CSK_PICK
    return nullptr;
}

// Smallest instantiated (rows per warp, float4 per lane) covering the shape.
bool reg_shape(int rows_per_cta, int n, int* rpw, int* cpl) {
    if (n % 4 != 0) return false;
    const int need_c = (n / 4 + 31) / 32;
    const int need_r = (rows_per_cta + kWarps - 1) / kWarps;
    const int cs[] = {1, 2, 4};
    const int rs[] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10};
    for (int c : cs) {
        if (c < need_c) continue;
        for (int r : rs) {
            if (r < need_r) continue;
            if (reg_kernel(r, c)) { *rpw = r; *cpl = c; return true; }
        }
        return false;
    }
    return false;
}

// ------------------------------------------------ GEMV path, streamed rows
// FP32 variant for rows that fit neither registers nor shared memory (MWRK on
// A itself, Remark 1, or a large sketch).  Every step streams the CTA's rows
// from HBM through a ring of up to kMaxStreamStages shared-memory blocks of
// kWarps * RPB rows, each filled by bulk copies (TMA, cp.async.bulk) that
// complete on the block's `full` mbarrier; the eight warps release a block on
// its `empty` mbarrier.  Thread 0 refills a stage one block after the CTA
// left it (no producer warp, so the CTA barriers of the reduction and the
// exchange see every thread), and tops the ring up before each exchange: the
// rows are the same every step, so the next step's first blocks load while
// this step's exchange runs.  Warp w scores rows w, w + kWarps, ... of each
// block against its register copy of x (lane l holds float4 columns l,
// l + 32, ...) with the register variant's arithmetic, order included, so
// the two give identical iterates.  Needs n % 4 == 0, n <= 128 * CPL, a
// leading dimension that is a multiple of 4 floats and 16-byte aligned rows.
#ifndef CSK_STREAM_MAX_STAGES
#define CSK_STREAM_MAX_STAGES 8
#endif
constexpr int kMaxStreamStages = CSK_STREAM_MAX_STAGES;   // ring depth: as many as fit, up to this
constexpr uint32_t kStreamWait = 1u << 24;      // try_wait polls per bulk-copy wait

// A 16-byte chunk of a row: four floats or two doubles.
template <typename T> struct Chunk;
template <> struct Chunk<float> {
    static constexpr int V = 4;
    using vec = float4;
    __device__ static void get(const vec& v, float (&e)[4]) { e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w; }
    __device__ static vec put(const float (&e)[4]) { return make_float4(e[0], e[1], e[2], e[3]); }
};
template <> struct Chunk<double> {
    static constexpr int V = 2;
    using vec = double2;
    __device__ static void get(const vec& v, double (&e)[2]) { e[0] = v.x; e[1] = v.y; }
    __device__ static vec put(const double (&e)[2]) { return make_double2(e[0], e[1]); }
};

// Rows per warp per block: a block holds kWarps * RPB rows of at most
// 32 * CPL chunks (<= 32 KB).  FP64 rows of up to 32 chunks (64 columns) take
// 8 rows per warp: the transposed sums and the scoring then serve 8 rows per
// warp instruction (FP64 instructions cost the same whatever the lanes hold).
template <typename T, int CPL>
struct StreamShape {
    static constexpr int RPB = (sizeof(T) == 8 && CPL == 1) ? 8 : (CPL <= 2 ? 4 : 8 / CPL);
    static constexpr int ROWS = kWarps * RPB;
};

// Shared memory: the ring, then bt and the row weights of the CTA's rows, and
// with UPD the stored residuals of those rows.
size_t stream_smem_bytes(int R, int n, int esize, int rows_per_blk, int stages, bool upd) {
    return (size_t)stages * rows_per_blk * n * esize + (size_t)(upd ? 3 : 2) * ((R + 3) & ~3) * esize;
}

// UPD: the residual-update form of Remark 1.  The CTA keeps r for its rows;
// a step takes the dot products of its rows with the previous step's chosen
// row At_{i} (kept in registers like x) instead of with x, and sets
// r_j = r_j - alpha * (At_j . At_i), r_i = 0 (exact arithmetic gives 0).  The
// first step, and every refresh_every-th, recomputes r = bt - At x.  Same
// bytes streamed per step as the GEMV form; only the dot products' second
// operand differs.
template <typename T, int CPL, bool UPD>
__global__ void __launch_bounds__(kIterThreads, 1)
k_iterate_gemv_stream(IterProblem p, int R, int nst) {
    constexpr int RPB = StreamShape<T, CPL>::RPB, SR = StreamShape<T, CPL>::ROWS;
    constexpr int V = Chunk<T>::V;
    using vec = typename Chunk<T>::vec;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ RedShared<T> sh;
    __shared__ __align__(8) uint64_t full[kMaxStreamStages];
    __shared__ __align__(8) uint64_t empty[kMaxStreamStages];
    int par = 0;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int n = p.n, d = p.d, nv = n / V;          // 16-byte chunks per row
    const int r0 = min(d, b * R), r1 = min(d, r0 + R), nr = r1 - r0;
    const int nblk = (nr + SR - 1) / SR;
    const size_t blk_elems = (size_t)SR * n;
    const uint32_t row_bytes = (uint32_t)n * sizeof(T);
    T* ring = reinterpret_cast<T*>(dsm);
    T* bts = ring + nst * blk_elems;
    T* w2s = bts + ((R + 3) & ~3);
    T* rst = w2s + ((R + 3) & ~3);            // UPD: the rows' residuals
    const T* At = static_cast<const T*>(p.At);
    const T* bt = static_cast<const T*>(p.bt);
    const T* x0 = static_cast<const T*>(p.x0);
    const T* xstar = static_cast<const T*>(p.xstar);
    const bool stat_owner = (b == 0 && warp == 0);
    const bool packed = p.ld == n;

    for (int q = tid; q < nr; q += blockDim.x) {
        bts[q] = bt[r0 + q];
        w2s[q] = weight_of<T>(p.N2[r0 + q]);
    }
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), kWarps);
        }
        mbar_fence_init();
    }
    __syncthreads();

    // Thread 0 only: blocks issued so far (block g holds row block g % nblk
    // in stage g % nst), and the stage, lap parity and row block of the next
    // issue; refill(upto) issues up to block `upto`, each stage taken over
    // once the warps released the block it held.
    int64_t issued = 0;
    int is = 0, iblk = 0;
    uint32_t ilap = 0;
    auto refill = [&](int64_t upto) -> bool {
        for (; issued < upto; ++issued) {
            if (issued >= nst && !mbar_wait(smem_u32(&empty[is]), ilap ^ 1u, kStreamWait))
                return false;
            const int q0 = iblk * SR, rows = min(SR, nr - q0);
            const uint32_t bar = smem_u32(&full[is]);
            const uint32_t dst = smem_u32(ring + is * blk_elems);
            mbar_expect_tx(bar, (uint32_t)rows * row_bytes);
            if (packed) {
                bulk_g2s(dst, At + (int64_t)(r0 + q0) * n, (uint32_t)rows * row_bytes, bar);
            } else {
                for (int q = 0; q < rows; ++q)
                    bulk_g2s(dst + (uint32_t)q * row_bytes, At + (int64_t)(r0 + q0 + q) * p.ld,
                             row_bytes, bar);
            }
            if (++iblk == nblk) iblk = 0;
            if (++is == nst) { is = 0; ilap ^= 1u; }
        }
        return true;
    };
    int stalled = 0;
    if (tid == 0 && nblk > 0 && !refill(nst)) stalled = 1;

    T xr[CPL][V], xsr[CPL][V], ar[CPL][V];   // ar (UPD): the previous step's chosen row
    T aprev = T(0);                           // UPD: its step length
    int32_t iprev = -1;                       //      and its row
#pragma unroll
    for (int i = 0; i < CPL; ++i) {
        const int c = lane + 32 * i;
#pragma unroll
        for (int e = 0; e < V; ++e) { xr[i][e] = T(0); xsr[i][e] = T(0); ar[i][e] = T(0); }
        if (x0 && c < nv) Chunk<T>::get(reinterpret_cast<const vec*>(x0)[c], xr[i]);
        if (xstar && c < nv) Chunk<T>::get(reinterpret_cast<const vec*>(xstar)[c], xsr[i]);
    }
    const T threshold = stop_threshold<T>(p.tol, *p.stop_norm, p.xstar ? p.n : p.d);
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    // chunk c of ||x - x*||^2 is counted by CTA c % G only: this lane's share
    // of the CPL chunks, fixed for the whole solve
    uint32_t stat_mask = 0;
#pragma unroll
    for (int i = 0; i < CPL; ++i)
        if (lane + 32 * i < nv && (lane + 32 * i) % (int)gridDim.x == b) stat_mask |= 1u << i;
    uint32_t round = 0;
    int64_t k = 0, g = 0;          // g: blocks consumed (the same count in every warp)
    int cs = 0;                    // stage of block g and its lap parity
    uint32_t clap = 0;
    int status = CSK_OK;
    int64_t next_fresh = 0;        // next recomputation step of the UPD form (0, K, 2K, ...)
    for (;;) {
        Red<T> c;
        c.key = T(-1); c.alpha = T(0); c.stat = T(0); c.idx = INT_MAX;
        // dot products against x (GEMV form, and the UPD form's recomputation
        // steps) or against the previous chosen row (UPD update steps)
        const bool fresh = k == next_fresh;
        if (fresh && p.refresh_every > 0) next_fresh += p.refresh_every;
        const bool use_x = !UPD || fresh;
        for (int blk = 0; blk < nblk && !stalled; ++blk, ++g) {
            const int s = cs;
            const uint32_t lap = clap;
            if (++cs == nst) { cs = 0; clap ^= 1u; }
            if (!mbar_wait(smem_u32(&full[s]), lap, kStreamWait)) {
                stalled = 1;
                break;
            }
            const T* rows = ring + s * blk_elems;
            const int q0 = blk * SR;
            T dot[RPB];
#pragma unroll
            for (int u = 0; u < RPB; ++u) {
                const vec* row = reinterpret_cast<const vec*>(rows + (size_t)(warp + kWarps * u) * n);
                const bool live = q0 + warp + kWarps * u < nr;
                T acc = T(0);
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const int cc = lane + 32 * i;
                    if (live && cc < nv) {
                        T a[V];
                        Chunk<T>::get(row[cc], a);
#pragma unroll
                        for (int e = 0; e < V; ++e) acc = fma(a[e], use_x ? xr[i][e] : ar[i][e], acc);
                    }
                }
                dot[u] = acc;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&empty[s]));
            {
                // lane l ends with row transpose_row(l) of the block and
                // keeps its own running candidate across the blocks
                const T sum = transpose_sum<T, RPB>(dot, lane);
                const int u = transpose_row<RPB>(lane);
                const int q = q0 + warp + kWarps * u;
                if (transpose_rep<RPB>(lane) && q < nr) {
                    T r;
                    if (!UPD || use_x) r = bts[q] - sum;
                    else r = (r0 + q == iprev) ? T(0) : fma(-aprev, sum, rst[q]);
                    if (UPD) rst[q] = r;
                    const T w = w2s[q];
                    if (!below_zero(w)) {
                        const T key = r * r * w;
                        if (better(key, r0 + q, c.key, c.idx)) { c.key = key; c.alpha = r * w; c.idx = r0 + q; }
                    }
                    if (!xstar) c.stat += r * r;
                }
            }
            // take over the stage of the previous block (released by now, as a rule)
            if (tid == 0 && !refill(g + nst)) stalled = 1;
        }
        // top the ring up: the next step's first blocks load during the exchange
        if (tid == 0 && nblk > 0 && !stalled && !refill(g + nst)) stalled = 1;
        if (__syncthreads_or(stalled)) {
            if (tid == 0) set_status_once(p.info, CSK_ETIMEOUT);
            status = CSK_ETIMEOUT;
            break;
        }
        if (xstar && warp == 0) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                if ((stat_mask >> i) & 1u) {
                    T t[V];
#pragma unroll
                    for (int e = 0; e < V; ++e) t[e] = xr[i][e] - xsr[i][e];
                    c.stat += chunk_sq(t);
                }
            }
        }
        c = block_reduce(c, sh, par);    // candidates differ across lanes
        if (!exchange(p.slots, round, c, spin, p.fault_inject, p.info, sh, par)) {
            status = CSK_ETIMEOUT;
            break;
        }
        ++round;
        const int dec = decide(c.stat, threshold, k, p.max_iter, c.key);
        if (dec != INT_MIN) { status = dec; break; }
        if (stat_owner && lane == 0 && p.ik_log && k < p.ik_log_len) p.ik_log[k] = c.idx;
        if (stat_owner && p.x_log && k < p.x_log_len)
#pragma unroll
            for (int i = 0; i < CPL; ++i)
                if (lane + 32 * i < nv)
                    reinterpret_cast<vec*>(static_cast<T*>(p.x_log) + k * n)[lane + 32 * i] =
                        Chunk<T>::put(xr[i]);
        const vec* arow = reinterpret_cast<const vec*>(At + (int64_t)c.idx * p.ld);
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int cc = lane + 32 * i;
            if (cc < nv) {
                T v[V];
                Chunk<T>::get(__ldg(arow + cc), v);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    xr[i][e] = fma(c.alpha, v[e], xr[i][e]);
                    if (UPD) ar[i][e] = v[e];
                }
            }
        }
        if (UPD) { aprev = c.alpha; iprev = c.idx; }
        ++k;
    }
    // no bulk copy may still be writing shared memory when the CTA exits
    if (tid == 0)
        for (int64_t q = g; q < issued; ++q) {
            (void)mbar_wait(smem_u32(&full[cs]), clap, kStreamWait);
            if (++cs == nst) { cs = 0; clap ^= 1u; }
        }
    if (stat_owner) {
        vec* xo = reinterpret_cast<vec*>(p.x_out);
#pragma unroll
        for (int i = 0; i < CPL; ++i)
            if (lane + 32 * i < nv) xo[lane + 32 * i] = Chunk<T>::put(xr[i]);
    }
    finish(p.info, status, k);
}

// Shared-memory GEMV loop: rows a warp scores in one pass, the smallest of
// 1, 2, 4, 8 covering its share of the CTA's rows (a transposed butterfly
// over N rows costs N + 4 adds, FP64 ones on the slow pipe).
// Rows a warp scores in one pass: FP32 spreads a CTA's rows over all its
// warps; FP64 packs up to kRowsPerWarp consecutive rows on each warp (see
// the loop's Phase A).
int gemv_rows_per_pass(int dtype, int rows_per_cta) {
    const int rpw = dtype == CSK_F64 ? rows_per_cta : (rows_per_cta + kWarps - 1) / kWarps;
    return rpw <= 1 ? 1 : rpw <= 2 ? 2 : rpw <= 4 ? 4 : kRowsPerWarp;
}

const void* gemv_kernel(int dtype, int rows_per_cta) {
    const int nr = gemv_rows_per_pass(dtype, rows_per_cta);
    const bool f64 = dtype == CSK_F64;
    switch (nr) {
        case 1: return f64 ? (const void*)k_iterate_gemv<double, 1> : (const void*)k_iterate_gemv<float, 1>;
        case 2: return f64 ? (const void*)k_iterate_gemv<double, 2> : (const void*)k_iterate_gemv<float, 2>;
        case 4: return f64 ? (const void*)k_iterate_gemv<double, 4> : (const void*)k_iterate_gemv<float, 4>;
        default: return f64 ? (const void*)k_iterate_gemv<double, 8> : (const void*)k_iterate_gemv<float, 8>;
    }
}

template <bool UPD>
const void* stream_kernel_t(int dtype, int cpl) {
    const bool f64 = dtype == CSK_F64;
    switch (cpl) {
        case 1: return f64 ? (const void*)k_iterate_gemv_stream<double, 1, UPD> : (const void*)k_iterate_gemv_stream<float, 1, UPD>;
        case 2: return f64 ? (const void*)k_iterate_gemv_stream<double, 2, UPD> : (const void*)k_iterate_gemv_stream<float, 2, UPD>;
        case 4: return f64 ? (const void*)k_iterate_gemv_stream<double, 4, UPD> : (const void*)k_iterate_gemv_stream<float, 4, UPD>;
        case 8: return f64 ? (const void*)k_iterate_gemv_stream<double, 8, UPD> : (const void*)k_iterate_gemv_stream<float, 8, UPD>;
        default: return nullptr;
    }
}

// Fused kernel of the shared-memory GEMV loop; vec: 16-byte loads of A in
// the sketch (A 16-byte aligned, n and lda multiples of the vector).
const void* fused_gemv_kernel(int dtype, int rows_per_cta, bool vec) {
    const int nr = gemv_rows_per_pass(dtype, rows_per_cta);
#define CSK_F(T, NR) (vec ? (const void*)k_fused_gemv<T, NR, (sizeof(T) == 8 ? 2 : 4), (sizeof(T) == 8 ? 2 : 4)> \
                         : (const void*)k_fused_gemv<T, NR, 1, 4>)
    if (dtype == CSK_F64)
        return nr == 1 ? CSK_F(double, 1) : nr == 2 ? CSK_F(double, 2) : nr == 4 ? CSK_F(double, 4)
                                                                         : CSK_F(double, 8);
    return nr == 1 ? CSK_F(float, 1) : nr == 2 ? CSK_F(float, 2) : nr == 4 ? CSK_F(float, 4)
                                                                   : CSK_F(float, 8);
#undef CSK_F
}

const void* stream_kernel(int dtype, int cpl, bool upd) {
    return upd ? stream_kernel_t<true>(dtype, cpl) : stream_kernel_t<false>(dtype, cpl);
}

int stream_rows_per_block(int dtype, int cpl) {
    const bool f64 = dtype == CSK_F64;
    switch (cpl) {
        case 1: return f64 ? StreamShape<double, 1>::ROWS : StreamShape<float, 1>::ROWS;
        case 2: return f64 ? StreamShape<double, 2>::ROWS : StreamShape<float, 2>::ROWS;
        case 4: return f64 ? StreamShape<double, 4>::ROWS : StreamShape<float, 4>::ROWS;
        case 8: return f64 ? StreamShape<double, 8>::ROWS : StreamShape<float, 8>::ROWS;
        default: return 0;
    }
}

// ------------------------------------------------------------ GRAM path
// Shared memory: r (Rpad) | w2 (Rpad) | x slice (spad) | x* slice (spad) |
// full x in FP64 for the refresh (npad doubles)
__global__ void __launch_bounds__(kIterThreads, 1)
k_iterate_gram(IterProblem p, int R) {
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ RedShared<float> sh;
    int par = 0;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int n = p.n, d = p.d;
    const int r0 = min(d, b * R), r1 = min(d, r0 + R), nr = r1 - r0;
    const int c0 = (int)((int64_t)n * b / G), c1 = (int)((int64_t)n * (b + 1) / G);
    const int Rpad = (R + 3) & ~3, spad = ((n + G - 1) / G + 4) & ~3;
    float* rs = reinterpret_cast<float*>(dsm);
    float* w2s = rs + Rpad;
    float* xsl = w2s + Rpad;
    float* xss = xsl + spad;
    double* xfull = reinterpret_cast<double*>(xss + spad);
    const float* At = static_cast<const float*>(p.At);
    const float* bt = static_cast<const float*>(p.bt);
    const float* x0 = static_cast<const float*>(p.x0);
    const float* xstar = static_cast<const float*>(p.xstar);
    float* xg = static_cast<float*>(p.xg);

    for (int c = c0 + tid; c < c1; c += blockDim.x) {
        xsl[c - c0] = x0 ? x0[c] : 0.0f;
        if (xstar) xss[c - c0] = xstar[c];
    }
    for (int q = tid; q < nr; q += blockDim.x) w2s[q] = weight_of<float>(p.N2[r0 + q]);
    __syncthreads();
    const float threshold = stop_threshold<float>(p.tol, *p.stop_norm, p.xstar ? p.n : p.d);
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    const int K = p.refresh_every;
    uint32_t round = 0;
    int64_t k = 0;
    int64_t next_refresh = 0;      // FP64 refresh steps 0, K, 2K, ... (no division per step)
    int status = CSK_OK;
    for (;;) {
        if (k == next_refresh) {
            if (K > 0) next_refresh += K;
            // FP64 refresh r = bt - At x: gather the x slices first; the
            // fence orders this CTA's slice stores before its slot words
            for (int c = c0 + tid; c < c1; c += blockDim.x) xg[c] = xsl[c - c0];
            __threadfence();
            __syncthreads();
            Red<float> dummy;
            dummy.key = -1.0f; dummy.alpha = 0.0f; dummy.stat = 0.0f; dummy.idx = INT_MAX;
            if (!exchange(p.slots, round, dummy, spin, p.fault_inject, p.info, sh, par, true)) {
                status = CSK_ETIMEOUT;
                break;
            }
            ++round;
            __threadfence();
            for (int c = tid; c < n; c += blockDim.x) xfull[c] = widen(__ldcg(xg + c));
            __syncthreads();
            // warp w sums the groups of kRefreshRows consecutive rows
            // w, w + kWarps, ... (FP32 entries widened exactly, FP64 FMA)
            for (int q0 = warp * kRefreshRows; q0 < nr; q0 += kWarps * kRefreshRows) {
                const int m = min(kRefreshRows, nr - q0);
                const double s = warp_rows_dot_f64<kRefreshRows>(At + (int64_t)(r0 + q0) * p.ld, p.ld, m,
                                                                 xfull, n, lane);
                const int u = transpose_row<kRefreshRows>(lane);
                if (transpose_rep<kRefreshRows>(lane) && u < m)
                    rs[q0 + u] = (float)(widen(bt[r0 + q0 + u]) - s);
            }
            __syncthreads();
        }
        // Phase A
        Red<float> c;
        c.key = -1.0f; c.alpha = 0.0f; c.stat = 0.0f; c.idx = INT_MAX;
        for (int q = tid; q < nr; q += blockDim.x) {
            const float r = rs[q], w = w2s[q];
            if (!(w < 0.0f)) {
                const float key = r * r * w;
                if (better(key, r0 + q, c.key, c.idx)) { c.key = key; c.alpha = r * w; c.idx = r0 + q; }
            }
            if (!xstar) c.stat += r * r;
        }
        if (xstar)
            for (int col = c0 + tid; col < c1; col += blockDim.x) {
                const float t = xsl[col - c0] - xss[col - c0];
                c.stat += t * t;
            }
        c = block_reduce(c, sh, par);
        RowPrefetch gpf;          // this CTA's slice of G[i_k, :], read from HBM after the exchange
        gpf.base = reinterpret_cast<const char*>(p.G + r0);
        gpf.ld = p.ldg * (int64_t)sizeof(float);
        gpf.bytes = nr * (int)sizeof(float) <= 32 * 128 ? nr * (int)sizeof(float) : 32 * 128;
        gpf.rows = d;
        if (!exchange(p.slots, round, c, spin, p.fault_inject, p.info, sh, par, false, gpf)) {
            status = CSK_ETIMEOUT;
            break;
        }
        ++round;
        const int dec = decide(c.stat, threshold, k, p.max_iter, c.key);
        if (dec != INT_MIN) { status = dec; break; }
        if (b == 0 && tid == 0 && p.ik_log && k < p.ik_log_len) p.ik_log[k] = c.idx;
        if (p.x_log && k < p.x_log_len)
            for (int col = c0 + tid; col < c1; col += blockDim.x)
                static_cast<float*>(p.x_log)[k * n + col] = xsl[col - c0];
        // r -= alpha G[i_k, :] on the owned rows, r_{i_k} = 0 exactly;
        // x slice += alpha At_{i_k}
        const float* grow = p.G + (int64_t)c.idx * p.ldg;
        for (int q = tid; q < nr; q += blockDim.x) {
            const int j = r0 + q;
            rs[q] = (j == c.idx) ? 0.0f : fmaf(-c.alpha, __ldg(grow + j), rs[q]);
        }
        const float* arow = At + (int64_t)c.idx * p.ld;
        for (int col = c0 + tid; col < c1; col += blockDim.x)
            xsl[col - c0] = fmaf(c.alpha, __ldg(arow + col), xsl[col - c0]);
        __syncthreads();
        ++k;
    }
    float* xo = static_cast<float*>(p.x_out);
    for (int col = c0 + tid; col < c1; col += blockDim.x) xo[col] = xsl[col - c0];
    finish(p.info, status, k);
}

// ------------------------------------------------ exchange floor probe
// `rounds` rounds of the register loop's per-step exchange -- the CTA
// reduction of a candidate, then the mailbox round trip with its reduction
// of the gathered candidates -- and no residual arithmetic.  The candidates
// are a cheap function of (CTA, thread, round), so the reductions do the
// same work as in a solve.
__global__ void __launch_bounds__(kIterThreads, 1)
k_exchange_probe(Slot* slots, int64_t rounds, csk_info* info) {
    __shared__ RedShared<float> sh;
    int par = 0;
    uint32_t round = 0;
    const uint32_t me = blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t k = 0; k < rounds; ++k) {
        Red<float> c;
        c.key = (float)((me * 2654435761u + (uint32_t)k * 40503u) >> 16);
        c.alpha = 1.0f;
        c.stat = 1.0f;
        c.idx = (int32_t)me;
        c = block_reduce(c, sh, par);
        if (!exchange(slots, round, c, kDefaultSpin, 0, info, sh, par)) break;
        ++round;
    }
}

// --------------------------------------------------------- final check
constexpr int kFinalThreads = 128;
constexpr int kFinalRows = 8;      // rows a warp sums at once in the final check

__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    return warp_sum(s);
}

template <typename T>
__global__ void __launch_bounds__(kFinalThreads)
k_final_rows(const T* __restrict__ At, int64_t ld, int d, int n, const T* __restrict__ bt,
             const double* __restrict__ N2, const T* __restrict__ x, double* __restrict__ part) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double rr = 0.0, bb = 0.0, empty = 0.0;
    // a warp takes kFinalRows consecutive rows at a time
    for (int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kFinalRows; j0 < d;
         j0 += nwarps * kFinalRows) {
        const int nr = (int)(d - j0 < kFinalRows ? d - j0 : kFinalRows);
        const double s = warp_rows_dot_f64<kFinalRows>(At + j0 * ld, ld, nr, x, n, lane);
        const int u = transpose_row<kFinalRows>(lane);
        if (transpose_rep<kFinalRows>(lane) && u < nr) {
            const int64_t j = j0 + u;
            const double bj = widen(bt[j]);
            const double r = bj - s;
            rr += r * r;
            bb += bj * bj;
            empty += (N2[j] > 0.0) ? 0.0 : 1.0;
        }
    }
    rr = block_sum_f64(rr, sh);
    bb = block_sum_f64(bb, sh);
    empty = block_sum_f64(empty, sh);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = rr;
        part[3 * blockIdx.x + 1] = bb;
        part[3 * blockIdx.x + 2] = empty;
    }
}

template <typename T>
__global__ void __launch_bounds__(kFinalThreads)
k_final_reduce(const double* __restrict__ part, int nparts, const T* __restrict__ x,
               const T* __restrict__ xstar, int n, csk_info* info) {
    __shared__ double sh[32];
    double rr = 0.0, bb = 0.0, empty = 0.0, ee = 0.0, ss = 0.0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) {
        rr += part[3 * t];
        bb += part[3 * t + 1];
        empty += part[3 * t + 2];
    }
    if (xstar)
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const double e = (double)x[c] - (double)xstar[c];
            ee += e * e;
            ss += (double)xstar[c] * (double)xstar[c];
        }
    rr = block_sum_f64(rr, sh);
    bb = block_sum_f64(bb, sh);
    empty = block_sum_f64(empty, sh);
    ee = block_sum_f64(ee, sh);
    ss = block_sum_f64(ss, sh);
    if (threadIdx.x == 0) {
        info->resid = sqrt(rr / bb);
        info->rse = xstar ? ee / ss : (double)NAN;
        info->empty_rows = (int32_t)empty;
    }
}

int final_blocks(int d) {
    DevInfo di;
    dev_info(&di);
    const int64_t rows_per_block = (int64_t)kFinalRows * (kFinalThreads / 32);
    int64_t blocks = ((int64_t)d + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)(di.sms > 0 ? di.sms : 1) * 4;
    return (int)(blocks < cap ? blocks : cap);
}

}  // namespace

// ------------------------------------------------------------ host side
int plan_iterate(int path, int dtype, int d, int n, int grid_req, int variant, bool vec_ok,
                 IterConfig* cfg) {
    DevInfo di;
    if (dev_info(&di) != 0) return CSK_ECUDA;
    const int s = dtype == CSK_F64 ? 8 : 4;
    const size_t budget = (size_t)di.smem_optin - 2048;   // static shared + slack
    int G = grid_req > 0 ? grid_req : di.sms;
    if (G > kMaxIterGrid) G = kMaxIterGrid;
    if (G > d) G = d;
    if (G < 1) G = 1;
    if (grid_req <= 0) {
        // small problems: fewer CTAs, cheaper exchange -- about 16K cells of
        // At per CTA in FP32, 1K in FP64 (this GPU's FP64 rate is 1/64 of
        // its FP32 rate, so a step's dot products need more SMs)
        const int64_t cells = (int64_t)d * n;
        const int64_t per_cta = dtype == CSK_F64 ? 1024 : 16384;
        int64_t want = (cells + per_cta - 1) / per_cta;
        if (want < 1) want = 1;
        if (want < G) G = (int)want;
    }
    const int R = (d + G - 1) / G;
    const int npad = (n + 3) & ~3, Rpad = (R + 3) & ~3, spad = ((n + G - 1) / G + 4) & ~3;
    cfg->grid = G;
    cfg->threads = kIterThreads;
    cfg->rows_per_cta = R;
    if (path == CSK_RESID_GRAM) {
        cfg->cache_rows = 0;
        cfg->smem = (size_t)(2 * Rpad + 2 * spad) * 4 + (size_t)npad * 8;
    } else {
        const size_t base = (size_t)(npad + 2 * Rpad + (dtype == CSK_F64 ? npad : spad)) * s;
        const size_t rows = (size_t)R * n * s;
        cfg->cache_rows = (base + rows <= budget) ? 1 : 0;
        cfg->smem = base + (cfg->cache_rows ? rows : 0);
    }
    cfg->reg_rpw = cfg->reg_cpl = 0;
    if (path == CSK_RESID_GEMV && dtype == CSK_F32 && vec_ok && variant != 1) {
        int rpw = 0, cpl = 0;
        if (reg_shape(R, n, &rpw, &cpl)) {
            cfg->reg_rpw = rpw;
            cfg->reg_cpl = cpl;
            cfg->cache_rows = 0;
            cfg->smem = 0;
        }
    }
    if (variant == 2 && cfg->reg_rpw == 0) return CSK_EUNSUPPORTED;
    // rows streamed through a bulk-copy ring: on request, or when the rows
    // stay resident neither in registers nor in shared memory; the
    // residual-update form (Remark 1) always runs this loop
    cfg->stream_cpl = 0;
    const int vlen = 16 / s;                 // elements per 16-byte chunk
    const bool upd = path == CSK_RESID_UPDATE;
    if (upd) cfg->reg_rpw = cfg->reg_cpl = 0;
    if ((upd || path == CSK_RESID_GEMV) && vec_ok && n % vlen == 0 &&
        (upd || variant == 3 || (variant == 0 && cfg->reg_rpw == 0 && !cfg->cache_rows))) {
        const int need_c = (n / vlen + 31) / 32;
        const int cpl = need_c <= 1 ? 1 : need_c <= 2 ? 2 : need_c <= 4 ? 4 : need_c <= 8 ? 8 : 0;
        int nst = kMaxStreamStages;
        while (cpl && nst > 2 &&
               stream_smem_bytes(R, n, s, stream_rows_per_block(dtype, cpl), nst, upd) > budget)
            --nst;
        const size_t sm = cpl ? stream_smem_bytes(R, n, s, stream_rows_per_block(dtype, cpl), nst, upd) : 0;
        if (cpl && sm <= budget) {
            cfg->stream_cpl = cpl;
            cfg->stream_stages = nst;
            cfg->reg_rpw = cfg->reg_cpl = 0;
            cfg->cache_rows = 0;
            cfg->smem = sm;
        }
    }
    if ((variant == 3 || upd) && cfg->stream_cpl == 0) return CSK_EUNSUPPORTED;
    if (cfg->smem > budget) return CSK_EUNSUPPORTED;
    return CSK_OK;
}

cudaError_t launch_iterate(int path, const IterProblem& p, const IterConfig& cfg, cudaStream_t st) {
    void* fn;
    const bool reg = cfg.reg_rpw > 0;
    const bool stream = cfg.stream_cpl > 0;
    if (path == CSK_RESID_GRAM) fn = (void*)k_iterate_gram;
    else if (stream) fn = const_cast<void*>(stream_kernel(p.dtype, cfg.stream_cpl,
                                                          path == CSK_RESID_UPDATE));
    else if (reg) fn = const_cast<void*>(reg_kernel(cfg.reg_rpw, cfg.reg_cpl));
    else fn = const_cast<void*>(gemv_kernel(p.dtype, cfg.rows_per_cta));
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_attr(fn, cfg.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cached_occupancy(fn, cfg.threads, cfg.smem, &per_sm);
    if (e != cudaSuccess) return e;
    DevInfo di;
    dev_info(&di);
    if ((int64_t)per_sm * di.sms < cfg.grid) return cudaErrorCooperativeLaunchTooLarge;
    IterProblem pc = p;
    int R = cfg.rows_per_cta, cache = cfg.cache_rows, nst = cfg.stream_stages;
    void* args_gemv[] = {&pc, &R, &cache};
    void* args_gram[] = {&pc, &R};
    void* args_stream[] = {&pc, &R, &nst};
    e = cudaLaunchCooperativeKernel(fn, dim3(cfg.grid), dim3(cfg.threads),
                                    stream ? args_stream
                                           : (path == CSK_RESID_GRAM || reg) ? args_gram : args_gemv,
                                    cfg.smem, st);
    if (e == cudaSuccess) note_launches(1);
    return e;
}

cudaError_t launch_exchange_probe(int grid, int64_t rounds, Slot* slots, csk_info* info,
                                  cudaStream_t st) {
    const void* fn = (const void*)k_exchange_probe;
    int per_sm = 0;
    cudaError_t e = cached_occupancy(fn, kIterThreads, 0, &per_sm);
    if (e != cudaSuccess) return e;
    DevInfo di;
    if (dev_info(&di) != 0) return cudaErrorUnknown;
    if ((int64_t)per_sm * di.sms < grid) return cudaErrorCooperativeLaunchTooLarge;
    void* args[] = {&slots, &rounds, &info};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kIterThreads), args, 0, st);
    if (e == cudaSuccess) note_launches(1);
    return e;
}

int plan_fused(int dtype, int64_t m, int d, int n, const IterConfig& cfg, const void* A,
               int64_t lda, int* cap, size_t* smem) {
    if (d > 65535 || m > (int64_t)INT_MAX / 2) return CSK_EUNSUPPORTED;
    if (cfg.stream_cpl > 0 || cfg.rows_per_cta > kOwnMaxBuckets) return CSK_EUNSUPPORTED;
    DevInfo di;
    if (dev_info(&di) != 0) return CSK_ECUDA;
    const int vl = dtype == CSK_F64 ? 2 : 4;
    const bool vec = reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % vl == 0 && n % vl == 0;
    if (cfg.reg_rpw > 0 && (!vec || cfg.reg_cpl != 4)) return CSK_EUNSUPPORTED;
    // row lists: 1.5 x the mean rows per CTA, within the shared memory left
    const size_t budget = (size_t)di.smem_optin - 2048 - sizeof(OwnShared);
    int64_t c = (3 * (m / cfg.grid) / 2 + 511) / 256 * 256;
    if (c < 1024) c = 1024;
    if (c > 16384) c = 16384;
    while (c > 256 && (size_t)c * 8 > budget) c -= 256;
    *cap = (int)c;
    *smem = cfg.smem > (size_t)c * 8 ? cfg.smem : (size_t)c * 8;
    if (*smem > budget) return CSK_EUNSUPPORTED;
    return CSK_OK;
}

cudaError_t launch_fused(int dtype, const IterProblem& p, const IterConfig& cfg,
                         const FusedArgs& fa, int cap, size_t smem, cudaStream_t st) {
    const int vl = dtype == CSK_F64 ? 2 : 4;
    const bool vec = reinterpret_cast<uintptr_t>(fa.A) % 16 == 0 && fa.lda % vl == 0 &&
                     p.n % vl == 0;
    const bool reg = cfg.reg_rpw > 0;
    void* fn = const_cast<void*>(reg ? fused_reg_kernel(cfg.reg_rpw, cfg.reg_cpl)
                                     : fused_gemv_kernel(dtype, cfg.rows_per_cta, vec));
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = ensure_smem_attr(fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cached_occupancy(fn, cfg.threads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    DevInfo di;
    dev_info(&di);
    if ((int64_t)per_sm * di.sms < cfg.grid) return cudaErrorCooperativeLaunchTooLarge;
    IterProblem pc = p;
    FusedSketch f;
    f.A = fa.A; f.lda = fa.lda; f.m = fa.m; f.b = fa.b; f.seed = fa.seed;
    f.h = fa.h; f.perm = fa.perm; f.off = fa.off; f.part = fa.part; f.cap = cap;
    int R = cfg.rows_per_cta, cache = cfg.cache_rows;
    void* args_reg[] = {&pc, &f, &R};
    void* args_gemv[] = {&pc, &f, &R, &cache};
    e = cudaLaunchCooperativeKernel(fn, dim3(cfg.grid), dim3(cfg.threads), reg ? args_reg : args_gemv,
                                    smem, st);
    if (e == cudaSuccess) note_launches(1);
    return e;
}

size_t final_check_partials(int d) { return (size_t)3 * final_blocks(d); }

cudaError_t launch_final_check(int dtype, const void* At, int64_t ld, int d, int n, const void* bt,
                               const double* N2, const void* x, const void* xstar, double* partials,
                               csk_info* info, cudaStream_t st) {
    const int blocks = final_blocks(d);
    if (dtype == CSK_F64) {
        k_final_rows<double><<<blocks, kFinalThreads, 0, st>>>((const double*)At, ld, d, n,
                                                               (const double*)bt, N2,
                                                               (const double*)x, partials);
        k_final_reduce<double><<<1, kFinalThreads, 0, st>>>(partials, blocks, (const double*)x,
                                                             (const double*)xstar, n, info);
    } else {
        k_final_rows<float><<<blocks, kFinalThreads, 0, st>>>((const float*)At, ld, d, n,
                                                              (const float*)bt, N2,
                                                              (const float*)x, partials);
        k_final_reduce<float><<<1, kFinalThreads, 0, st>>>(partials, blocks, (const float*)x,
                                                            (const float*)xstar, n, info);
    }
    note_launches(2);
    return cudaGetLastError();
}

}  // namespace csk
