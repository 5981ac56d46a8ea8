// own_sketch.cuh -- the bucket-owner count sketch (Algorithm 1, Initialize:
// At = S A, bt = S b with S = Phi D of Definition 1) as device code for one
// CTA, shared by the sketch kernel (csk_sketch) and the fused sketch-and-loop
// kernels (csk_solve with fused = 1).
//
// Every row's bucket h(i) is stored first in 16 bits (hash16_range, d <=
// 65535).  A CTA that owns the contiguous buckets [j0, j1) then does
// everything for them (own_sketch_cta):
//   1. scans h (16-byte loads, L2-resident): counts the rows of every owned
//      bucket and the rows of all earlier buckets (= its first offset), and
//      lists its own rows (shared-memory atomics);
//   2. places them by bucket and ranks them inside the bucket by row index,
//      so each bucket's rows are in ascending order, the sign D_ii riding in
//      bit 31 -- and writes off and perm for its range;
//   3. warp w sums buckets j0 + w, j0 + w + W, ... over all columns, rows in
//      ascending order, several rows' 16-byte loads in flight per lane, then
//      ||At_j||^2 in FP64 and bt_j.
// No kernel-wide synchronisation and no per-bucket barrier.  The additions
// are those of the counting-sort path (0 + s_0 a_0 + s_1 a_1 + ... in
// ascending row order), so At and bt are the same bits.  When a CTA's rows
// exceed its shared-memory list (cap), it handles its buckets in sub-ranges
// that fit, rescanning h for each; a bucket larger than cap is put in order
// by a stable ballot compaction of one warp over h and summed by all warps
// over column chunks.
#pragma once

#include <climits>
#include <cstdint>

#include "common.cuh"

namespace csk {

template <typename T, int V> struct VecOf;
template <> struct VecOf<float, 4> { using type = float4; };
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<double, 2> { using type = double2; };
template <> struct VecOf<double, 1> { using type = double; };

template <typename T, int V>
__device__ __forceinline__ void vload(const T* p, T (&out)[V]) {
    using VT = typename VecOf<T, V>::type;
    VT v = __ldg(reinterpret_cast<const VT*>(p));
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int q = 0; q < V; ++q) out[q] = e[q];
}

template <typename T, int V>
__device__ __forceinline__ void vstore(T* p, const T (&in)[V]) {
    using VT = typename VecOf<T, V>::type;
    VT v;
    T* e = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int q = 0; q < V; ++q) e[q] = in[q];
    *reinterpret_cast<VT*>(p) = v;
}

constexpr int kOwnMaxWarps = 16;          // warps of a CTA running own_sketch_cta, at most
constexpr int kOwnMaxBuckets = 1024;      // buckets one CTA owns at most

// h[i] = h(i) for i = first, first + step, ... in groups of 8 (16-byte
// stores); `first` and `step` count groups of 8 rows.
__device__ __forceinline__ void hash16_range(int64_t m, uint32_t d, uint64_t seed,
                                             uint16_t* __restrict__ h, int64_t first,
                                             int64_t step) {
    for (int64_t i0 = first * 8; i0 < m; i0 += step * 8) {
        uint16_t v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            v[q] = i0 + q < m ? (uint16_t)row_bucket(row_hash(seed, (uint64_t)(i0 + q)), d) : 0;
        if (i0 + 8 <= m) {
            uint4 t;
            t.x = v[0] | ((uint32_t)v[1] << 16);
            t.y = v[2] | ((uint32_t)v[3] << 16);
            t.z = v[4] | ((uint32_t)v[5] << 16);
            t.w = v[6] | ((uint32_t)v[7] << 16);
            *reinterpret_cast<uint4*>(h + i0) = t;
        } else {
            for (int q = 0; i0 + q < m; ++q) h[i0 + q] = v[q];
        }
    }
}

struct OwnShared {
    int cnt[kOwnMaxBuckets];
    int loc[kOwnMaxBuckets + 1];
    int fill[kOwnMaxBuckets];
    int below_w[kOwnMaxWarps];
    double part[kOwnMaxWarps];
    int nlist;
};

// One warp: the signed sum of the rows rows[a..c) (in that order) of src over
// the column chunks cfirst, cfirst + cstep, ... (32 V CPL columns each) into
// dst; returns this lane's FP64 sum of squares of the values it wrote.  With
// EMB the sign of a row rides in bit 31 of its entry, else it is recomputed
// from the hash.  U rows (32 registers of loads per lane) are loaded before
// any is added.
template <typename T, int V, int CPL, bool EMB>
__device__ __forceinline__ double own_sum(const T* __restrict__ src, int64_t ld, int ncols,
                                          const int32_t* rows, int a, int c, uint64_t seed,
                                          T* __restrict__ dst, int cfirst, int cstep) {
    constexpr int W32 = (int)(sizeof(T) / 4) * V * CPL;     // 32-bit registers per row
    constexpr int U = 32 / W32 < 1 ? 1 : 32 / W32;
    const int lane = lane_id();
    double sq = 0.0;
    for (int c0 = cfirst; c0 < ncols; c0 += cstep) {
        T acc[CPL][V];
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc)
#pragma unroll
            for (int q = 0; q < V; ++q) acc[cc][q] = T(0);
        for (int q0 = a; q0 < c; q0 += U) {
            T vals[U][CPL][V];
            bool neg[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = q0 + u < c;
                const int32_t e = ok ? rows[q0 + u] : 0;
                const int32_t row = EMB ? (e & 0x7fffffff) : e;
                neg[u] = EMB ? (e < 0) : (ok && row_negative(row_hash(seed, (uint64_t)row)));
                const T* rp = src + (int64_t)row * ld;
#pragma unroll
                for (int cc = 0; cc < CPL; ++cc) {
                    const int col = c0 + (cc * 32 + lane) * V;
                    if (ok && col < ncols) {
                        vload<T, V>(rp + col, vals[u][cc]);
                    } else {
#pragma unroll
                        for (int q = 0; q < V; ++q) vals[u][cc][q] = T(0);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (q0 + u < c) {
#pragma unroll
                    for (int cc = 0; cc < CPL; ++cc)
#pragma unroll
                        for (int q = 0; q < V; ++q)
                            acc[cc][q] = neg[u] ? acc[cc][q] - vals[u][cc][q] : acc[cc][q] + vals[u][cc][q];
                }
        }
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
            const int col = c0 + (cc * 32 + lane) * V;
            if (col < ncols) {
                vstore<T, V>(dst + col, acc[cc]);
#pragma unroll
                for (int q = 0; q < V; ++q) sq += (double)acc[cc][q] * (double)acc[cc][q];
            }
        }
    }
    return sq;
}

// One warp: bt_j = sum of the signed b values of rows[a..c) in that order
// (one right-hand side); every lane returns the sum.
template <typename T, bool EMB>
__device__ __forceinline__ T own_sum_b1(const T* __restrict__ B, int64_t ldb, const int32_t* rows,
                                        int a, int c, uint64_t seed) {
    const int lane = lane_id();
    T acc = T(0);
    for (int q0 = a; q0 < c; q0 += 32) {
        const bool ok = q0 + lane < c;
        const int32_t e = ok ? rows[q0 + lane] : 0;
        const int32_t row = EMB ? (e & 0x7fffffff) : e;
        const bool neg = EMB ? (e < 0) : (ok && row_negative(row_hash(seed, (uint64_t)row)));
        T v = ok ? B[(int64_t)row * ldb] : T(0);
        if (neg) v = -v;
        const int cnt = min(32, c - q0);
        for (int t = 0; t < cnt; ++t) acc += __shfl_sync(0xffffffffu, v, t);
    }
    return acc;
}

// Buckets [ka, kb) of this CTA whose rows (relative to base = loc[ka]) are
// listed in ascending order with their signs in `list`: warp w sums buckets
// ka + w, ka + w + W, ...
template <typename T, int V, int CPL>
__device__ __forceinline__ void own_sum_range(const T* __restrict__ A, int64_t lda, int n,
                                              const T* __restrict__ B, int64_t ldb, int nrhs,
                                              const int32_t* list, const OwnShared& sh, int ka,
                                              int kb, int j0, uint64_t seed, T* __restrict__ At,
                                              T* __restrict__ Bt, double* __restrict__ N2) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    constexpr int CW = 32 * V * CPL;
    const int base = sh.loc[ka];
    for (int k = ka + warp; k < kb; k += W) {
        const int a = sh.loc[k] - base, c = sh.loc[k + 1] - base;
        const int64_t j = j0 + k;
        double sq = own_sum<T, V, CPL, true>(A, lda, n, list, a, c, seed, At + j * n, 0, CW);
        sq = warp_sum(sq);
        if (lane == 0 && N2) N2[j] = sq;
        if (B && nrhs == 1) {
            const T bs = own_sum_b1<T, true>(B, ldb, list, a, c, seed);
            if (lane == 0) Bt[j] = bs;
        } else if (B) {
            (void)own_sum<T, 1, 1, true>(B, ldb, nrhs, list, a, c, seed, Bt + j * nrhs, 0, 32);
        }
    }
}

// One CTA (all its threads; at most kOwnMaxWarps warps): the sketch of the
// buckets [j0, j1) (j1 - j0 <= kOwnMaxBuckets), from h (every row's bucket,
// complete and visible), with a shared-memory row list of cap entries in
// `list` and `ord` each.  Writes At, Bt (nullable), N2 (nullable) for those
// buckets, off[j0 .. j1) (and off[d] = m when j1 == d) and perm over their
// rows (perm is also the storage of a bucket larger than cap, so it is
// required).  h is read with coherent (L2) loads: it may have been written
// earlier in the same kernel.
template <typename T, int V, int CPL>
__device__ __forceinline__ void own_sketch_cta(const T* __restrict__ A, int64_t lda, int n,
                                               int64_t m, const T* __restrict__ B, int64_t ldb,
                                               int nrhs, const uint16_t* h, int d,
                                               uint64_t seed, int cap, T* __restrict__ At,
                                               T* __restrict__ Bt, double* __restrict__ N2,
                                               int32_t* __restrict__ perm, int32_t* __restrict__ off,
                                               int j0, int j1, int32_t* list, int32_t* ord,
                                               OwnShared& sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = blockDim.x, W = nt >> 5;
    const int nb = j1 - j0;
    for (int k = tid; k < nb; k += nt) { sh.cnt[k] = 0; sh.fill[k] = 0; }
    if (tid == 0) sh.nlist = 0;
    __syncthreads();

    // 1. count (and list) the owned rows; rows of earlier buckets give the offset.
    // Each thread issues kScanLoads 16-byte loads before looking at any, so a
    // CTA's scan of h costs a few L2 round trips, not one per load.
    constexpr int kScanLoads = 8;
    int below = 0;
    auto take = [&](int64_t i0, const uint4& t) {
        const uint16_t v[8] = {(uint16_t)(t.x & 0xFFFF), (uint16_t)(t.x >> 16),
                               (uint16_t)(t.y & 0xFFFF), (uint16_t)(t.y >> 16),
                               (uint16_t)(t.z & 0xFFFF), (uint16_t)(t.z >> 16),
                               (uint16_t)(t.w & 0xFFFF), (uint16_t)(t.w >> 16)};
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int hv = v[q];               // 0xFFFF is no bucket: d <= 65535
            if (hv < j0) {
                ++below;
            } else if (hv < j1) {
                atomicAdd(&sh.cnt[hv - j0], 1);
                const int p = atomicAdd(&sh.nlist, 1);
                if (p < cap) list[p] = (int32_t)(i0 + q);
            }
        }
    };
    const int64_t m8 = m / 8;                  // whole 16-byte groups
    const uint4* h4 = reinterpret_cast<const uint4*>(h);
    for (int64_t g0 = tid; g0 < m8; g0 += (int64_t)nt * kScanLoads) {
        uint4 t[kScanLoads];
#pragma unroll
        for (int u = 0; u < kScanLoads; ++u) {
            const int64_t g = g0 + (int64_t)u * nt;
            t[u] = g < m8 ? __ldcg(h4 + g) : make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu,
                                                       0xFFFFFFFFu);
        }
#pragma unroll
        for (int u = 0; u < kScanLoads; ++u) take((g0 + (int64_t)u * nt) * 8, t[u]);
    }
    if (tid == 0 && m8 * 8 < m) {              // the last m % 8 rows
        uint16_t v[8];
        for (int q = 0; q < 8; ++q) v[q] = m8 * 8 + q < m ? __ldcg(h + m8 * 8 + q) : (uint16_t)0xFFFF;
        take(m8 * 8, make_uint4(v[0] | ((uint32_t)v[1] << 16), v[2] | ((uint32_t)v[3] << 16),
                                v[4] | ((uint32_t)v[5] << 16), v[6] | ((uint32_t)v[7] << 16)));
    }
    below = warp_sum(below);
    if (lane == 0) sh.below_w[warp] = below;
    __syncthreads();
    below = 0;
    for (int w = 0; w < W; ++w) below += sh.below_w[w];
    // exclusive scan of the counts (warp 0; lane l takes a contiguous run)
    if (warp == 0) {
        const int per = (nb + 31) / 32;
        int s = 0;
        for (int t = 0; t < per; ++t) {
            const int k = lane * per + t;
            if (k < nb) s += sh.cnt[k];
        }
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - s;
        for (int t = 0; t < per; ++t) {
            const int k = lane * per + t;
            if (k < nb) { sh.loc[k] = run; run += sh.cnt[k]; }
        }
        if (lane == 31) sh.loc[nb] = incl;
    }
    __syncthreads();
    const int total = sh.loc[nb];
    for (int k = tid; k < nb; k += nt) off[j0 + k] = below + sh.loc[k];
    if (j1 == d && tid == 0) off[d] = (int32_t)m;

    if (total <= cap) {
        // 2. place by bucket, then rank inside the bucket by row index
        for (int e = tid; e < total; e += nt) {
            const int32_t i = list[e];
            const int k = (int)__ldcg(h + i) - j0;
            ord[sh.loc[k] + atomicAdd(&sh.fill[k], 1)] = i;
        }
        __syncthreads();
        for (int e = tid; e < total; e += nt) {
            const int32_t i = ord[e];
            const int k = (int)__ldcg(h + i) - j0;
            const int a = sh.loc[k], c = sh.loc[k + 1];
            int rank = 0;
            for (int q = a; q < c; ++q) rank += ord[q] < i;
            const bool neg = row_negative(row_hash(seed, (uint64_t)i));
            list[a + rank] = neg ? (int32_t)((uint32_t)i | 0x80000000u) : i;
            perm[below + a + rank] = i;
        }
        __syncthreads();
        // 3. sums
        own_sum_range<T, V, CPL>(A, lda, n, B, ldb, nrhs, list, sh, 0, nb, j0, seed, At, Bt, N2);
        return;
    }
    // the rows do not fit the list: sub-ranges of buckets that fit
    int ka = 0;
    while (ka < nb) {
        if (sh.cnt[ka] > cap) {
            // one bucket larger than the list: warp 0 writes its rows to perm
            // in ascending order (stable ballot compaction over h); all warps
            // then sum column chunks of it, rows read back from perm
            const int a = sh.loc[ka], c = sh.loc[ka + 1];
            const int jb = j0 + ka;
            int32_t* prow = perm + below + a;
            if (warp == 0) {
                int written = 0;
                for (int64_t i0 = 0; i0 < m; i0 += 32) {
                    const int64_t i = i0 + lane;
                    const bool hit = i < m && (int)__ldcg(h + i) == jb;
                    const unsigned bal = __ballot_sync(0xffffffffu, hit);
                    if (hit) prow[written + __popc(bal & lanemask_lt())] = (int32_t)i;
                    written += __popc(bal);
                }
            }
            __syncthreads();
            constexpr int CW = 32 * V * CPL;
            const double sq = warp_sum(own_sum<T, V, CPL, false>(A, lda, n, prow, 0, c - a, seed,
                                                              At + (int64_t)jb * n, warp * CW,
                                                              W * CW));
            if (B && nrhs > 1)
                (void)own_sum<T, 1, 1, false>(B, ldb, nrhs, prow, 0, c - a, seed,
                                           Bt + (int64_t)jb * nrhs, warp * 32, W * 32);
            if (lane == 0) sh.part[warp] = sq;
            if (B && nrhs == 1 && warp == 0) {
                const T bs = own_sum_b1<T, false>(B, ldb, prow, 0, c - a, seed);
                if (lane == 0) Bt[jb] = bs;
            }
            __syncthreads();
            if (tid == 0 && N2) {
                double t = 0.0;
                for (int w = 0; w < W; ++w) t += sh.part[w];
                N2[jb] = t;
            }
            ++ka;
            continue;
        }
        int kb = ka + 1;
        while (kb < nb && sh.cnt[kb] <= cap && sh.loc[kb + 1] - sh.loc[ka] <= cap) ++kb;
        const int base = sh.loc[ka], lo = j0 + ka, hi = j0 + kb;
        for (int64_t i = tid; i < m; i += nt) {
            const int hv = __ldcg(h + i);
            if (hv >= lo && hv < hi) {
                const int k = hv - j0;
                ord[sh.loc[k] - base + atomicAdd(&sh.fill[k], 1)] = (int32_t)i;
            }
        }
        __syncthreads();
        const int cntr = sh.loc[kb] - base;
        for (int e = tid; e < cntr; e += nt) {
            const int32_t i = ord[e];
            const int k = (int)__ldcg(h + i) - j0;
            const int a = sh.loc[k] - base, c = sh.loc[k + 1] - base;
            int rank = 0;
            for (int q = a; q < c; ++q) rank += ord[q] < i;
            const bool neg = row_negative(row_hash(seed, (uint64_t)i));
            list[a + rank] = neg ? (int32_t)((uint32_t)i | 0x80000000u) : i;
            perm[below + base + a + rank] = i;
        }
        __syncthreads();
        own_sum_range<T, V, CPL>(A, lda, n, B, ldb, nrhs, list, sh, ka, kb, j0, seed, At, Bt, N2);
        __syncthreads();
        ka = kb;
    }
}

}  // namespace csk
