// sketch.cu -- count sketch formation At = S A, bt = S b (Algorithm 1,
// "Initialize"; S = Phi D of Definition 1) on sm_103a.
//
// Pipeline (all integer work bit-exact, FP work in a fixed order):
//   k_hist        cnt[j] = #{i : h(i) = j}, and row i's slot in its bucket
//                 (warp-aggregated atomics)
//   k_scan_*      off = exclusive prefix sum of cnt   (off[d] = m)
//   k_scatter     perm_tmp[off[h(i)] + slot(i)] = i: rows grouped by bucket
//                 (in the atomics' order inside a bucket)
//   k_segsum      resident CTAs claim buckets: each puts a bucket's rows in
//                 ascending order in shared memory (writing perm, the rows in
//                 (h(i), i) order -- unique, so independent of the atomics'
//                 order), then At_j = sum_{p in bucket j, ascending} D_ii A_i
//                 and ||At_j||^2 in FP64: a warp per column chunk (128
//                 columns in FP32; up to 256, sized to the row, in FP64),
//                 16-byte loads, 4 (narrow FP64 rows: 8) rows in flight
//   k_segsum_warp the same sums for FP32 with at most 128 rows per bucket on
//                 average and enough buckets to occupy the warps: a warp per
//                 bucket over up to 512 columns at once, ordered by
//                 shuffles, no CTA barrier; bt as well for one right-hand side
//   k_segsum_b1   bt likewise, FP64 with one right-hand side, a warp per 8
//                 buckets
//   k_segsum_b    Bt likewise otherwise, a warp per bucket
// The kernels after k_hist launch with programmatic stream serialization and
// wait for their predecessor inside (pdl_wait).
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "fp64.cuh"
#include "kernels.h"
#include "own_sketch.cuh"

#ifndef CSK_SKETCH_PDL
#define CSK_SKETCH_PDL 1
#endif

namespace csk {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096 buckets per tile
constexpr int kScanSingle = kScanThreads * 32;   // one-block scan up to 32768 buckets (R <= 8)
constexpr int kSortCap = 1024;           // rows of a bucket ordered in shared memory

inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Launch with programmatic stream serialization: the kernel may be scheduled
// before its predecessor in the stream has finished, and waits for it inside
// (pdl_wait), which hides the launch gap between the short kernels of the
// sketch.
template <typename... KArgs, typename... Args>
cudaError_t launch_dep(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = CSK_SKETCH_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ------------------------------------------------------------- histogram
// Bucket counts, and each row's slot among the rows of its bucket (in the
// order the atomics happen to run; the segmented sum orders every bucket by
// row index afterwards).  Lanes of a warp that share a bucket take
// consecutive slots from one atomic.
__global__ void k_hist(int64_t m, uint32_t d, uint64_t seed, int32_t* __restrict__ cnt,
                       int32_t* __restrict__ slot) {
    pdl_trigger();
    // warp-uniform trip count: every lane reaches the match below together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = lane_id();
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m;
         base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < m;
        const int32_t j = valid ? row_bucket(row_hash(seed, (uint64_t)i), d) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, j);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (valid && lane == leader) first = atomicAdd(&cnt[j], __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (valid) slot[i] = first + __popc(peers & lanemask_lt());
    }
}

// ------------------------------------------------------------------ scan
// Block-wide exclusive scan of kScanThreads * ITEMS int32 values starting at
// `first` (thread t takes ITEMS consecutive values).
template <int ITEMS>
__device__ __forceinline__ int block_scan_tile(const int32_t* __restrict__ cnt, int64_t first,
                                               int64_t d, int carry_in, int32_t* __restrict__ out,
                                               int* sh_warp) {
    const int t = threadIdx.x;
    const int64_t i0 = first + (int64_t)t * ITEMS;
    int v[ITEMS];
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) v[q] = (i0 + q < d) ? cnt[i0 + q] : 0;
    int run = 0;
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) run += v[q];
    // warp inclusive scan of the per-thread totals
    int w = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, w, o);
        if ((int)lane_id() >= o) w += y;
    }
    const int warp = t >> 5;
    if (lane_id() == 31) sh_warp[warp] = w;
    __syncthreads();
    if (warp == 0) {
        int s = (int)lane_id() < (kScanThreads / 32) ? sh_warp[lane_id()] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if ((int)lane_id() >= o) s += y;
        }
        sh_warp[lane_id()] = s;   // inclusive totals of warps
    }
    __syncthreads();
    const int warp_excl = warp ? sh_warp[warp - 1] : 0;
    const int base = carry_in + warp_excl + (w - run);
    int ex = base;
#pragma unroll
    for (int q = 0; q < ITEMS; ++q) {
        if (i0 + q < d) out[i0 + q] = ex;
        ex += v[q];
    }
    const int total = sh_warp[kScanThreads / 32 - 1];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_partials(const int32_t* __restrict__ cnt, int64_t d, int32_t* __restrict__ part) {
    pdl_wait();
    pdl_trigger();
    __shared__ int sh[32];
    const int64_t i0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) s += (i0 + q < d) ? cnt[i0 + q] : 0;
    s = warp_sum(s);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = sh[threadIdx.x];
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const int32_t* __restrict__ cnt, int64_t d, const int32_t* __restrict__ part,
             int32_t* __restrict__ off) {
    pdl_wait();
    pdl_trigger();
    __shared__ int sh[32];
    __shared__ int carry;
    // carry-in of this tile: sum of the partials of the tiles before it
    int s = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) s += part[t];
    s = warp_sum(s);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = sh[threadIdx.x];
        v = warp_sum(v);
        if (threadIdx.x == 0) carry = v;
    }
    __syncthreads();
    const int c = carry;
    __syncthreads();
    const int total = block_scan_tile<kScanItems>(cnt, (int64_t)blockIdx.x * kScanTile, d, c, off, sh);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) off[d] = c + total;
}

// The whole scan in one block of kScanThreads, for d <= kScanSingle.  Warp w
// owns the contiguous segment [128 R w, 128 R (w + 1)) and reads it in R
// coalesced rounds of 128 counts (4 per lane); each round is scanned across
// the warp with shuffles and carried into the next, then the warps' totals
// are scanned in shared memory.
template <int R>
__global__ void __launch_bounds__(kScanThreads)
k_scan_single(const int32_t* __restrict__ cnt, int64_t d, int32_t* __restrict__ off) {
    pdl_wait();
    pdl_trigger();
    __shared__ int wsum[kScanThreads / 32];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int64_t seg = (int64_t)warp * 128 * R;
    int v[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = seg + 128 * r + 4 * lane;
        if (i + 3 < d) {
            const int4 t = *reinterpret_cast<const int4*>(cnt + i);
            v[r][0] = t.x; v[r][1] = t.y; v[r][2] = t.z; v[r][3] = t.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[r][q] = i + q < d ? cnt[i + q] : 0;
        }
    }
    int excl[R];
    int carry = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int t = v[r][0] + v[r][1] + v[r][2] + v[r][3];
        int sc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += y;
        }
        excl[r] = carry + sc - t;
        carry += __shfl_sync(0xffffffffu, sc, 31);
    }
    if (lane == 0) wsum[warp] = carry;
    __syncthreads();
    if (warp == 0) {
        const int t = wsum[lane];
        int sc = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += y;
        }
        wsum[lane] = sc - t;                       // exclusive offset of warp `lane`
        if (lane == 31) off[d] = sc;               // total
    }
    __syncthreads();
    const int base = wsum[warp];
    const bool vec_out = (reinterpret_cast<uintptr_t>(off) & 15) == 0;   // off may be the caller's
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = seg + 128 * r + 4 * lane;
        int e[4];
        e[0] = base + excl[r];
        e[1] = e[0] + v[r][0];
        e[2] = e[1] + v[r][1];
        e[3] = e[2] + v[r][2];
        if (vec_out && i + 3 < d) {
            *reinterpret_cast<int4*>(off + i) = make_int4(e[0], e[1], e[2], e[3]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i + q < d) off[i + q] = e[q];
        }
    }
}

// --------------------------------------------------------------- scatter
// Row i goes to perm_tmp[off[h(i)] + slot[i]]: no atomics, the slots were
// taken by the histogram pass.
__global__ void k_scatter(int64_t m, uint32_t d, uint64_t seed, const int32_t* __restrict__ slot,
                          const int32_t* __restrict__ off, int32_t* __restrict__ perm_tmp) {
    pdl_wait();
    pdl_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t j = row_bucket(row_hash(seed, (uint64_t)i), d);
        perm_tmp[off[j] + slot[i]] = (int32_t)i;
    }
}

// ------------------------------------------------- segmented row sum
// Signed sum of the rows perm[p0..p1) of src, columns [c0, c0 + 32 V CPL)
// of ncols, into dst, by one warp, ascending p in every column.  Returns this
// lane's sum of squares of its finished columns (FP64).
template <typename T, int V, int CPL, int U>
__device__ __forceinline__ double seg_chunk(const T* __restrict__ src, int64_t ld, int ncols, int c0,
                                            const int32_t* __restrict__ perm, int32_t p0,
                                            int32_t p1, uint64_t seed, T* __restrict__ dst) {
    const int lane = lane_id();
    T acc[CPL][V];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int q = 0; q < V; ++q) acc[c][q] = T(0);
    for (int32_t pb = p0; pb < p1; pb += 32) {
        const int32_t myrow = (pb + lane < p1) ? perm[pb + lane] : 0;
        const int myneg = row_negative(row_hash(seed, (uint64_t)myrow)) ? 1 : 0;
        const int cnt = min(32, p1 - pb);
        for (int q0 = 0; q0 < cnt; q0 += U) {
            T vals[U][CPL][V];
            int neg[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t row = __shfl_sync(0xffffffffu, myrow, (q0 + u) & 31);
                neg[u] = __shfl_sync(0xffffffffu, myneg, (q0 + u) & 31);
                const bool valid = q0 + u < cnt;
                const T* rp = src + (int64_t)row * ld;
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int col = c0 + (c * 32 + lane) * V;
                    if (valid && col < ncols) {
                        vload<T, V>(rp + col, vals[u][c]);
                    } else {
#pragma unroll
                        for (int q = 0; q < V; ++q) vals[u][c][q] = T(0);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q0 + u < cnt) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c)
#pragma unroll
                        for (int q = 0; q < V; ++q)
                            acc[c][q] = neg[u] ? acc[c][q] - vals[u][c][q] : acc[c][q] + vals[u][c][q];
                }
            }
        }
    }
    double sq = 0.0;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int col = c0 + (c * 32 + lane) * V;
        if (col < ncols) {
            vstore<T, V>(dst + col, acc[c]);
#pragma unroll
            for (int q = 0; q < V; ++q) sq += (double)acc[c][q] * (double)acc[c][q];
        }
    }
    return sq;
}

// Resident CTAs claim buckets one at a time from a counter.  The bucket's rows, grouped but in no
// particular order by the scatter, are ranked by row index in shared memory
// (rows are distinct, so every rank is unique) and written to perm in
// ascending order; a bucket larger than kSortCap is regenerated in ascending
// order by a stable compaction over all rows instead (O(m), only for d far
// below m / kSortCap).  Then warp w sums the column chunks w, w + W, ... of
// the bucket's rows in that order; the FP64 row norm is combined across
// warps in a fixed order.
template <typename T, int V, int CPL, int U>
// 10 CTAs per SM in FP32 (48 registers; at 56 the kernel ran markedly slower), 7 in FP64;
// the one-warp FP64 variants for narrow (U = 8) or 129..256-column rows
// (CPL > 2) get room for their loads
__global__ void __launch_bounds__(128, (U > 4 || CPL * V > 4) ? 4 : (sizeof(T) == 4 ? 10 : 7))
k_segsum(const T* __restrict__ A, int64_t lda, int n, int64_t m,
         const int32_t* __restrict__ perm_tmp, int32_t* __restrict__ perm,
         const int32_t* __restrict__ off, int d, uint64_t seed, T* __restrict__ At,
         double* __restrict__ N2, int32_t* __restrict__ next) {
    pdl_wait();
    pdl_trigger();
    __shared__ double part[4];
    __shared__ __align__(16) int32_t ubuf[kSortCap];
    __shared__ __align__(16) int32_t sbuf[kSortCap];
    constexpr int CW = 32 * V * CPL;                 // columns per chunk
    const int tid = threadIdx.x, nt = blockDim.x;
    const int W = nt >> 5, warp = tid >> 5, lane = lane_id();
    __shared__ int32_t claim;
    for (;;) {
        // the next unclaimed bucket: every CTA stays busy until the last ones
        if (tid == 0) claim = atomicAdd(next, 1);
        __syncthreads();
        const int64_t j = claim;
        if (j >= d) break;
        const int32_t p0 = off[j], p1 = off[j + 1], cnt = p1 - p0;
        const int32_t* rows = sbuf;
        int32_t q0 = 0;
        if (cnt <= kSortCap) {
            for (int t = tid; t < cnt; t += nt) ubuf[t] = perm_tmp[p0 + t];
            __syncthreads();
            for (int t = tid; t < cnt; t += nt) {
                const int32_t v = ubuf[t];
                int rank = 0;
                int q = 0;
                for (; q + 4 <= cnt; q += 4) {
                    const int4 u = *reinterpret_cast<const int4*>(ubuf + q);
                    rank += (u.x < v) + (u.y < v) + (u.z < v) + (u.w < v);
                }
                for (; q < cnt; ++q) rank += ubuf[q] < v;
                sbuf[rank] = v;
                perm[p0 + rank] = v;
            }
        } else {
            if (warp == 0) {
                int32_t written = 0;
                for (int64_t i0 = 0; i0 < m; i0 += 32) {
                    const int64_t i = i0 + lane;
                    const bool hit = i < m && row_bucket(row_hash(seed, (uint64_t)i), d) == (int32_t)j;
                    const unsigned bal = __ballot_sync(0xffffffffu, hit);
                    if (hit) perm[p0 + written + __popc(bal & lanemask_lt())] = (int32_t)i;
                    written += __popc(bal);
                }
            }
            rows = perm;
            q0 = p0;
        }
        __syncthreads();
        double sq = 0.0;
        for (int c0 = warp * CW; c0 < n; c0 += W * CW)
            sq += seg_chunk<T, V, CPL, U>(A, lda, n, c0, rows, q0, q0 + cnt, seed, At + j * (int64_t)n);
        sq = warp_sum(sq);
        if (lane == 0) part[warp] = sq;
        __syncthreads();
        if (tid == 0 && N2) {
            double t = 0.0;
            for (int w = 0; w < W; ++w) t += part[w];
            N2[j] = t;
        }
        __syncthreads();
    }
}

// Signed sums of the right-hand sides in ascending row order.
//
// FP64, one right-hand side (k_segsum_b1): a warp takes kBGroup buckets at a time
// and lane l < kBGroup sums bucket l of the group.  Each round the warp loads
// the next 32 rows of every bucket of the group (lane q takes row q of each,
// coalesced within a bucket), puts the signed values in a warp-private
// shared tile, and lanes 0..kBGroup-1 add their bucket's values in order.
// One add instruction thus serves kBGroup buckets: this GPU issues a warp's
// FP64 instruction at the same cost however few lanes are active.
//
// FP32 (k_segsum_b): one warp per bucket.  One right-hand side: the lanes
// load 32 rows' values at once and the sum takes them in order through
// shuffles.  Several: lanes over the columns, rows in order, 4 rows in
// flight.
constexpr int kBGroup = 8;
constexpr int kBWarps = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kBWarps)
k_segsum_b1(const T* __restrict__ B, int64_t ldb, const int32_t* __restrict__ perm,
            const int32_t* __restrict__ off, int d, uint64_t seed, T* __restrict__ Bt) {
    pdl_wait();
    __shared__ T tile[kBWarps][kBGroup][33];   // padded: lanes 0..7 read distinct banks
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * kBWarps;
    for (int64_t j0 = ((int64_t)blockIdx.x * kBWarps + warp) * kBGroup; j0 < d; j0 += nwarps * kBGroup) {
        // lane g <= kBGroup reads off[j0 + g]; bucket g of the group spans [p0_g, p0_{g+1})
        const int64_t jl = j0 + (lane <= kBGroup ? lane : kBGroup);
        const int32_t offl = off[jl < d ? jl : d];
        const int32_t mycnt = __shfl_down_sync(0xffffffffu, offl, 1) - offl;   // lanes < kBGroup
        int32_t p0[kBGroup], cnt[kBGroup];
        int32_t maxcnt = 0;
#pragma unroll
        for (int g = 0; g < kBGroup; ++g) {
            p0[g] = __shfl_sync(0xffffffffu, offl, g);
            cnt[g] = __shfl_sync(0xffffffffu, offl, g + 1) - p0[g];   // 0 past d
            maxcnt = max(maxcnt, cnt[g]);
        }
        T acc = T(0);
        for (int32_t pb = 0; pb < maxcnt; pb += 32) {
            int32_t row[kBGroup];
#pragma unroll
            for (int g = 0; g < kBGroup; ++g) row[g] = pb + lane < cnt[g] ? perm[p0[g] + pb + lane] : -1;
#pragma unroll
            for (int g = 0; g < kBGroup; ++g) {
                T v = T(0);
                if (row[g] >= 0) {
                    v = B[(int64_t)row[g] * ldb];
                    if (row_negative(row_hash(seed, (uint64_t)row[g]))) v = -v;
                }
                tile[warp][g][lane] = v;
            }
            __syncwarp();
            if (lane < kBGroup) {
                const int32_t c = min(32, mycnt - pb);
                for (int q = 0; q < c; ++q) acc += tile[warp][lane][q];
            }
            __syncwarp();
        }
        if (lane < kBGroup && j0 + lane < d) Bt[j0 + lane] = acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_segsum_b(const T* __restrict__ B, int64_t ldb, int nrhs, const int32_t* __restrict__ perm,
           const int32_t* __restrict__ off, int d, uint64_t seed, T* __restrict__ Bt) {
    pdl_wait();
    const int lane = lane_id();
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < d; j += nwarps) {
        const int32_t p0 = off[j], p1 = off[j + 1];
        if (nrhs == 1) {
            T acc = T(0);
            for (int32_t pb = p0; pb < p1; pb += 32) {
                const bool valid = pb + lane < p1;
                const int32_t row = valid ? perm[pb + lane] : 0;
                T v = valid ? B[(int64_t)row * ldb] : T(0);
                if (row_negative(row_hash(seed, (uint64_t)row))) v = -v;
                const int cnt = min(32, p1 - pb);
                for (int q = 0; q < cnt; ++q) acc += __shfl_sync(0xffffffffu, v, q);
            }
            if (lane == 0) Bt[j] = acc;
        } else {
            for (int c0 = 0; c0 < nrhs; c0 += 32)
                (void)seg_chunk<T, 1, 1, 4>(B, ldb, nrhs, c0, perm, p0, p1, seed, Bt + j * (int64_t)nrhs);
        }
    }
}

// ------------------------------------------ warp-per-bucket segmented sum
// FP32 sketches whose buckets hold at most kWarpMean rows on average: each
// warp claims a bucket of its own and runs it through without a CTA barrier,
// so one warp's claim, ordering and final sums overlap the other warps' row
// loads (with 20 to 50 rows per bucket those fixed steps are a large part of
// a bucket), and a lane keeps 32 values in flight across up to 512 columns
// (twice the CTA kernel's 16 over 128) at 60 to 68 registers.  A bucket of
// at most kWarpCap rows is ordered in registers (lane l holds rows l and
// l + 32 of the scatter's order and counts, by shuffles, how many of the
// bucket's rows are smaller: its rank); the ordered rows go to a
// warp-private list in shared memory and to perm.  A larger bucket is
// ranked against perm_tmp in global memory and read back from perm.  Then
// the warp sums every column chunk of the bucket in ascending row order (the
// same additions as k_segsum) and, with one right-hand side, bt_j as
// k_segsum_b does: the signed values of the rows added in ascending order,
// their loads issued before the column pass and consumed after it.
constexpr int kWarpCap = 64;
constexpr int kWarpMean = 128;
constexpr int kWarpThreads = 128;

template <int V, int CPL, int U>
__global__ void __launch_bounds__(kWarpThreads, CPL >= 4 ? 7 : 8)
k_segsum_warp(const float* __restrict__ A, int64_t lda, int n, const int32_t* __restrict__ perm_tmp,
              int32_t* __restrict__ perm, const int32_t* __restrict__ off, int d, uint64_t seed,
              float* __restrict__ At, double* __restrict__ N2, int32_t* __restrict__ next,
              const float* __restrict__ B, int64_t ldb, float* __restrict__ Bt) {
    pdl_wait();
    pdl_trigger();
    __shared__ __align__(16) int32_t list[kWarpThreads / 32][kWarpCap];
    constexpr int CW = 32 * V * CPL;                 // columns per chunk
    const int lane = lane_id();
    int32_t* my = list[threadIdx.x >> 5];
    for (;;) {
        int32_t j = 0;
        if (lane == 0) j = atomicAdd(next, 1);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= d) break;
        const int32_t p0 = off[j], cnt = off[j + 1] - p0;
        const bool small = cnt <= kWarpCap;
        const int32_t* rows = my;
        int32_t q0 = 0;
        if (small) {
            const int32_t v0 = lane < cnt ? perm_tmp[p0 + lane] : INT_MAX;
            const int32_t v1 = lane + 32 < cnt ? perm_tmp[p0 + 32 + lane] : INT_MAX;
            int r0 = 0, r1 = 0;
            const int c32 = cnt < 32 ? cnt : 32;
            for (int q = 0; q < c32; ++q) {
                const int32_t u = __shfl_sync(0xffffffffu, v0, q);
                r0 += u < v0;
                r1 += u < v1;
            }
            for (int q = 32; q < cnt; ++q) {
                const int32_t u = __shfl_sync(0xffffffffu, v1, q - 32);
                r0 += u < v0;
                r1 += u < v1;
            }
            if (lane < cnt) {
                my[r0] = v0;
                perm[p0 + r0] = v0;
            }
            if (lane + 32 < cnt) {
                my[r1] = v1;
                perm[p0 + r1] = v1;
            }
        } else {
            for (int t = lane; t < cnt; t += 32) {
                const int32_t v = perm_tmp[p0 + t];
                int rank = 0;
                for (int q = 0; q < cnt; ++q) rank += perm_tmp[p0 + q] < v;
                perm[p0 + rank] = v;
            }
            rows = perm;
            q0 = p0;
        }
        __syncwarp();
        float b0 = 0.f, b1 = 0.f;
        if (Bt && small) {
            if (lane < cnt) {
                const int32_t r = my[lane];
                b0 = B[(int64_t)r * ldb];
                if (row_negative(row_hash(seed, (uint64_t)r))) b0 = -b0;
            }
            if (lane + 32 < cnt) {
                const int32_t r = my[lane + 32];
                b1 = B[(int64_t)r * ldb];
                if (row_negative(row_hash(seed, (uint64_t)r))) b1 = -b1;
            }
        }
        double sq = 0.0;
        for (int c0 = 0; c0 < n; c0 += CW)
            sq += seg_chunk<float, V, CPL, U>(A, lda, n, c0, rows, q0, q0 + cnt, seed, At + (int64_t)j * n);
        sq = warp_sum(sq);
        if (lane == 0 && N2) N2[j] = sq;
        if (Bt) {
            float acc = 0.f;
            if (small) {
                const int c32 = cnt < 32 ? cnt : 32;
                for (int q = 0; q < c32; ++q) acc += __shfl_sync(0xffffffffu, b0, q);
                for (int q = 32; q < cnt; ++q) acc += __shfl_sync(0xffffffffu, b1, q - 32);
            } else {
                for (int32_t pb = 0; pb < cnt; pb += 32) {
                    const bool valid = pb + lane < cnt;
                    const int32_t r = valid ? rows[q0 + pb + lane] : 0;
                    float v = valid ? B[(int64_t)r * ldb] : 0.f;
                    if (row_negative(row_hash(seed, (uint64_t)r))) v = -v;
                    const int c = min(32, cnt - pb);
                    for (int q = 0; q < c; ++q) acc += __shfl_sync(0xffffffffu, v, q);
                }
            }
            if (lane == 0) Bt[j] = acc;
        }
        __syncwarp();   // the list is rewritten for the next bucket
    }
}

// --------------------------------------------- bucket-owner sketch (FP32)
// FP32 sketches whose buckets are small (at most kOwnMaxMean rows on
// average, d <= 65535) and whose A is at most kOwnMaxElems elements skip the
// global counting sort (own_sketch.cuh): k_hash16 stores every row's bucket
// in 16 bits, then CTA b of k_sketch_own owns the contiguous buckets
// [d b / G, d (b + 1) / G) and orders and sums them itself.
constexpr int kOwnThreads = 512;
constexpr int kOwnMaxMean = 128;          // mean rows per bucket of this path
constexpr int64_t kOwnMaxElems = 32ll << 20;   // elements of A of this path (by default)
constexpr int kOwnMaxCap = 16384;         // rows a CTA lists in shared memory at most
constexpr int64_t kOwnWarpElems = 4ll << 20;   // elements of A from which the warp-per-bucket sum may win

__global__ void k_hash16(int64_t m, uint32_t d, uint64_t seed, uint16_t* __restrict__ h) {
    hash16_range(m, d, seed, h, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (int64_t)gridDim.x * blockDim.x);
}

template <int V, int CPL>
__global__ void __launch_bounds__(kOwnThreads, 1)
k_sketch_own(const float* __restrict__ A, int64_t lda, int n, int64_t m,
             const float* __restrict__ B, int64_t ldb, int nrhs, const uint16_t* h,
             int d, uint64_t seed, int cap, float* __restrict__ At, float* __restrict__ Bt,
             double* __restrict__ N2, int32_t* __restrict__ perm, int32_t* __restrict__ off) {
    extern __shared__ __align__(16) int32_t own_dsm[];
    __shared__ OwnShared sh;
    pdl_wait();                         // h comes from the hash pass
    const int G = gridDim.x, b = blockIdx.x;
    const int j0 = (int)((int64_t)d * b / G), j1 = (int)((int64_t)d * (b + 1) / G);
    own_sketch_cta<float, V, CPL>(A, lda, n, m, B, ldb, nrhs, h, d, seed, cap, At, Bt, N2, perm,
                                  off, j0, j1, own_dsm, own_dsm + cap, sh);
}

// ----------------------------------------------------------- row norms
// A warp takes kNormRows consecutive rows at a time; per row the squares of
// columns lane, lane + 32, ... accumulate in order (FMA), then a butterfly.
constexpr int kNormRows = 8;

template <typename T>
__global__ void k_row_norms(const T* __restrict__ A, int64_t ld, int rows, int n,
                            double* __restrict__ N2) {
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = lane_id();
    for (int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kNormRows;
         j0 < rows; j0 += nwarps * kNormRows) {
        const int nr = (int)(rows - j0 < kNormRows ? rows - j0 : kNormRows);
        const double s = warp_rows_sq_f64<kNormRows>(A + j0 * ld, ld, nr, n, lane);
        const int u = transpose_row<kNormRows>(lane);
        if (transpose_rep<kNormRows>(lane) && u < nr) N2[j0 + u] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_norm2(const T* __restrict__ v, int64_t len, double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const double t = (double)v[i];
        s += t * t;
    }
    s = warp_sum(s);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) out[0] = t;
    }
}

}  // namespace

// ------------------------------------------------------------ host side
size_t sort_scratch_bytes(int64_t m, int64_t d) {
    const int64_t tiles = (d + kScanTile - 1) / kScanTile;
    return (size_t)(align_up(4 * (d + 1), 256) + align_up(4 * (d + 1), 256) + 2 * align_up(4 * m, 256) +
                    align_up(4 * tiles, 256));
}

void carve_sort_scratch(void* base, int64_t m, int64_t d, SortScratch* s) {
    char* p = static_cast<char*>(base);
    const int64_t tiles = (d + kScanTile - 1) / kScanTile;
    s->cnt = reinterpret_cast<int32_t*>(p);       p += align_up(4 * (d + 1), 256);
    s->off = reinterpret_cast<int32_t*>(p);       p += align_up(4 * (d + 1), 256);
    s->perm_tmp = reinterpret_cast<int32_t*>(p);  p += align_up(4 * m, 256);
    s->perm = reinterpret_cast<int32_t*>(p);      p += align_up(4 * m, 256);
    s->part = reinterpret_cast<int32_t*>(p);      p += align_up(4 * tiles, 256);
    (void)p;
}

cudaError_t launch_bucket_group(int64_t m, int64_t d, uint64_t seed, const SortScratch& s,
                                cudaStream_t st) {
    DevInfo di;
    if (dev_info(&di) != 0) return cudaErrorUnknown;
    cudaError_t e = cudaMemsetAsync(s.cnt, 0, (size_t)(d + 1) * 4, st);   // counts and the claim counter
    if (e != cudaSuccess) return e;
    const int threads = 256;
    int64_t blocks = (m + threads - 1) / threads;
    if (blocks > (int64_t)di.sms * 16) blocks = (int64_t)di.sms * 16;
    // the slots live in perm until the segmented sum writes the sorted rows there
    k_hist<<<(int)blocks, threads, 0, st>>>(m, (uint32_t)d, seed, s.cnt, s.perm);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (d <= kScanSingle) {
        // rounds of 128 counts per warp: 32 warps x 128 R >= d
        const int64_t need = (d + 32 * 128 - 1) / (32 * 128);
        auto fn = need <= 1 ? k_scan_single<1> : need <= 2 ? k_scan_single<2>
                : need <= 4 ? k_scan_single<4> : k_scan_single<8>;
        e = launch_dep(fn, 1, kScanThreads, st, s.cnt, d, s.off);
        note_launches(3);
    } else {
        const int64_t tiles = (d + kScanTile - 1) / kScanTile;
        e = launch_dep(k_scan_partials, (int)tiles, kScanThreads, st, s.cnt, d, s.part);
        if (e == cudaSuccess)
            e = launch_dep(k_scan_tiles, (int)tiles, kScanThreads, st, s.cnt, d, s.part, s.off);
        note_launches(4);
    }
    if (e == cudaSuccess)
        e = launch_dep(k_scatter, (int)blocks, threads, st, m, (uint32_t)d, seed, s.perm, s.off,
                       s.perm_tmp);
    return e;
}

namespace {
int sketch_path_override();

// Bt for the right-hand sides after the segmented sum of A has written perm.
cudaError_t launch_segsum_rhs(int dtype, const void* B, int64_t ldb, int nrhs, const SortScratch& s,
                              int d, uint64_t seed, void* Bt, const DevInfo& di, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (B && nrhs == 1 && dtype == CSK_F64) {
        int64_t bblocks = ((int64_t)d + kBWarps * kBGroup - 1) / (kBWarps * kBGroup);
        if (bblocks > (int64_t)di.sms * 32) bblocks = (int64_t)di.sms * 32;
        e = launch_dep(k_segsum_b1<double>, (int)bblocks, 32 * kBWarps, st, (const double*)B, ldb,
                       s.perm, s.off, d, seed, (double*)Bt);
        note_launches(1);
    } else if (B && nrhs > 0) {
        int64_t bblocks = ((int64_t)d + 7) / 8;
        if (bblocks > (int64_t)di.sms * 32) bblocks = (int64_t)di.sms * 32;
        if (dtype == CSK_F32)
            e = launch_dep(k_segsum_b<float>, (int)bblocks, 256, st, (const float*)B, ldb, nrhs,
                           s.perm, s.off, d, seed, (float*)Bt);
        else
            e = launch_dep(k_segsum_b<double>, (int)bblocks, 256, st, (const double*)B, ldb, nrhs,
                           s.perm, s.off, d, seed, (double*)Bt);
        note_launches(1);
    }
    return e;
}

// FP32: the warp-per-bucket kernel for the row layout.  32 values a lane in
// flight (8 16-byte, 16 8-byte or 32 4-byte loads), over up to 512 columns
// at once.
using WarpSegsumFn = decltype(&k_segsum_warp<4, 1, 8>);
WarpSegsumFn pick_segsum_warp(const float* A, int64_t lda, int n) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(A);
    const bool vec = (a % 16 == 0) && (lda % 4 == 0) && (n % 4 == 0);
    const bool vec2 = (a % 8 == 0) && (lda % 2 == 0) && (n % 2 == 0);   // 8-byte loads
    if (vec) return n <= 128 ? k_segsum_warp<4, 1, 8> : n <= 256 ? k_segsum_warp<4, 2, 4> : k_segsum_warp<4, 4, 2>;
    if (vec2) return n <= 128 ? k_segsum_warp<2, 2, 8> : n <= 256 ? k_segsum_warp<2, 4, 4> : k_segsum_warp<2, 8, 2>;
    return k_segsum_warp<1, 4, 8>;
}

// Whether the warp-per-bucket kernel takes an FP32 sketch: buckets of at most
// kWarpMean rows on average, and at least half as many buckets as resident
// warps.  Measured on GB300 (whole sketch, one right-hand side): ahead of the
// CTA per bucket from 100000 x 100 to 1e6 x 1000 and up to 120 rows per
// bucket (300000 x 50, d = 2500), behind it with 1500 buckets for ~4000
// warps (30000 x 1000).  *fn and *per_sm return the kernel and its residency.
cudaError_t warp_segsum_fits(const float* A, int64_t lda, int64_t m, int n, int64_t d,
                             const DevInfo& di, WarpSegsumFn* fn, int* per_sm, bool* fits) {
    *fn = pick_segsum_warp(A, lda, n);
    *per_sm = 0;
    const cudaError_t e = cached_occupancy((const void*)*fn, kWarpThreads, 0, per_sm);
    if (e != cudaSuccess) return e;
    const int64_t warps = (int64_t)*per_sm * di.sms * (kWarpThreads / 32);
    *fits = m <= (int64_t)kWarpMean * d && 2 * d >= warps;
    return cudaSuccess;
}

// k_segsum_warp on per_sm resident CTAs a SM (their warps claim the
// buckets; at most one warp per bucket); it also sums bt for one right-hand
// side, k_segsum_b the others.
cudaError_t launch_segsum_warp(WarpSegsumFn fn, int per_sm, const float* A, int64_t lda, int n,
                               const float* B, int64_t ldb, int nrhs, const SortScratch& s, int d,
                               uint64_t seed, float* At, float* Bt, double* N2, const DevInfo& di,
                               cudaStream_t st) {
    const int64_t resident = (int64_t)(per_sm > 0 ? per_sm : 1) * di.sms;
    const int64_t need = ((int64_t)d + kWarpThreads / 32 - 1) / (kWarpThreads / 32);
    const int blocks = (int)(resident < need ? resident : need);
    const bool fold_b = B && nrhs == 1;
    cudaError_t e = launch_dep(fn, blocks, kWarpThreads, st, A, lda, n, s.perm_tmp, s.perm, s.off, d,
                               seed, At, N2, s.cnt + d, fold_b ? B : nullptr, ldb,
                               fold_b ? Bt : nullptr);
    note_launches(1);
    if (e == cudaSuccess && !fold_b)
        e = launch_segsum_rhs(CSK_F32, B, ldb, nrhs, s, d, seed, Bt, di, st);
    return e;
}
}  // namespace

cudaError_t launch_segsum(int dtype, const void* A, int64_t lda, int64_t m, int n, const void* B,
                          int64_t ldb, int nrhs, const SortScratch& s, int d, uint64_t seed,
                          void* At, void* Bt, double* N2, cudaStream_t st) {
    DevInfo di;
    if (dev_info(&di) != 0) return cudaErrorUnknown;
    const uintptr_t a = reinterpret_cast<uintptr_t>(A);
    // FP32: a warp per bucket where warp_segsum_fits says so.  Forced, it
    // still needs buckets of at most kWarpMean rows on average: a bucket
    // above kWarpCap rows is ranked in O(rows^2 / 32) steps per warp.
    const int o = sketch_path_override();
    if (dtype == CSK_F32 && o != 4) {
        WarpSegsumFn wf;
        int per_sm = 0;
        bool fits = false;
        cudaError_t e = warp_segsum_fits(static_cast<const float*>(A), lda, m, n, d, di, &wf, &per_sm, &fits);
        if (e != cudaSuccess) return e;
        if (o == 3 ? m <= (int64_t)kWarpMean * d : fits)
            return launch_segsum_warp(wf, per_sm, static_cast<const float*>(A), lda, n,
                                      static_cast<const float*>(B), ldb, nrhs, s, d, seed,
                                      static_cast<float*>(At), static_cast<float*>(Bt), N2, di, st);
    }
    // warps per bucket: one per column chunk, at most 4.  FP32: 128-column
    // chunks.  FP64 adds occupy the slow pipe at the same cost whatever the
    // lanes hold, so an FP64 row of up to 256 columns is one chunk sized to
    // it (no chunk half made of zeros), and a row of at most 64 columns keeps
    // 8 rows in flight instead of 4 (a warp moves few bytes per row).
    int cw = 128;
    const void* fn = nullptr;
    if (dtype == CSK_F32) {
        const bool vec = (a % 16 == 0) && (lda % 4 == 0) && (n % 4 == 0);
        const bool vec2 = (a % 8 == 0) && (lda % 2 == 0) && (n % 2 == 0);   // 8-byte loads
        fn = vec ? (const void*)k_segsum<float, 4, 1, 4>
           : vec2 ? (const void*)k_segsum<float, 2, 2, 4> : (const void*)k_segsum<float, 1, 4, 4>;
    } else {
        const bool vec = (a % 16 == 0) && (lda % 2 == 0) && (n % 2 == 0);
        if (vec) {
            const int c2 = (n + 63) / 64;                 // double2 chunks per lane to cover the row
            fn = c2 <= 1 ? (const void*)k_segsum<double, 2, 1, 8>
               : c2 == 2 ? (const void*)k_segsum<double, 2, 2, 4>
               : c2 == 3 ? (const void*)k_segsum<double, 2, 3, 4>
               : c2 == 4 ? (const void*)k_segsum<double, 2, 4, 4> : (const void*)k_segsum<double, 2, 2, 4>;
            cw = c2 <= 4 ? 64 * (c2 < 1 ? 1 : c2) : 128;
        } else {
            fn = n <= 64 ? (const void*)k_segsum<double, 1, 2, 8> : (const void*)k_segsum<double, 1, 4, 4>;
            cw = n <= 64 ? 64 : 128;
        }
    }
    const int warps = (n + cw - 1) / cw < 1 ? 1 : ((n + cw - 1) / cw > 4 ? 4 : (n + cw - 1) / cw);
    const int bs = 32 * warps;
    // as many CTAs as stay resident (they claim the buckets), at most d
    int per_sm = 0;
    cudaError_t e = cached_occupancy(fn, bs, 0, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t resident = (int64_t)(per_sm > 0 ? per_sm : 1) * di.sms;
    const int blocks = (int)(resident < d ? resident : d);
    if (dtype == CSK_F32)
        e = launch_dep(reinterpret_cast<decltype(&k_segsum<float, 4, 1, 4>)>(const_cast<void*>(fn)), blocks,
                       bs, st, (const float*)A, lda, n, m, s.perm_tmp, s.perm, s.off, d, seed, (float*)At,
                       N2, s.cnt + d);
    else
        e = launch_dep(reinterpret_cast<decltype(&k_segsum<double, 2, 2, 4>)>(const_cast<void*>(fn)), blocks,
                       bs, st, (const double*)A, lda, n, m, s.perm_tmp, s.perm, s.off, d, seed,
                       (double*)At, N2, s.cnt + d);
    note_launches(1);
    if (e == cudaSuccess) e = launch_segsum_rhs(dtype, B, ldb, nrhs, s, d, seed, Bt, di, st);
    return e;
}

namespace {
// Test and measurement hooks read once from the environment: CSK_SKETCH_PATH
// = "sort" or "own" forces the counting-sort or the bucket-owner FP32 path
// (where the owner path applies), "warp" or "cta" the counting sort with the
// warp-per-bucket (where buckets hold at most kWarpMean rows on average) or
// the CTA-per-bucket segmented sum (FP32; FP64 always takes the CTA one);
// CSK_SKETCH_OWN_CAP caps a CTA's row list (exercises the sub-range and
// large-bucket code of the owner path).
int env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}
int sketch_path_override() {
    static const int p = [] {
        const char* v = getenv("CSK_SKETCH_PATH");
        if (!v) return 0;
        if (!strcmp(v, "sort")) return 1;
        if (!strcmp(v, "own")) return 2;
        if (!strcmp(v, "warp")) return 3;
        if (!strcmp(v, "cta")) return 4;
        return 0;
    }();
    return p;
}

bool use_owner_path(int dtype, const void* A, int64_t lda, int64_t m, int64_t n, int64_t d,
                    int nrhs) {
    if (dtype != CSK_F32 || d > 65535 || m > (int64_t)INT_MAX / 2) return false;
    const int o = sketch_path_override();
    if (o == 2) return true;
    if (o != 0) return false;
    // measured on GB300: ahead of the counting sort with the CTA-per-bucket
    // sum up to ~25M elements of A (fixed costs of the sort chain dominate
    // there), behind it at 100000 x 500 with one right-hand side and above
    if (!(m <= (int64_t)kOwnMaxMean * d && m * (int64_t)n <= kOwnMaxElems)) return false;
    // with at most one right-hand side and from kOwnWarpElems elements of A,
    // the sort chain with the warp-per-bucket sum is ahead where it applies
    // (100000 x 100, d = 5000: 31 against 47 us; 300000 x 100, d = 10000: 55
    // against 104; 20000 x 100, d = 1000: even)
    if (nrhs > 1 || m * (int64_t)n < kOwnWarpElems) return true;
    DevInfo di;
    if (dev_info(&di) != 0) return true;
    WarpSegsumFn wf;
    int per_sm = 0;
    bool fits = false;
    if (warp_segsum_fits(static_cast<const float*>(A), lda, m, (int)n, d, di, &wf, &per_sm, &fits) !=
        cudaSuccess)
        return true;
    return !fits;
}

cudaError_t launch_sketch_own(const float* A, int64_t lda, int64_t m, int n, const float* B,
                              int64_t ldb, int nrhs, const SortScratch& s, int d, uint64_t seed,
                              float* At, float* Bt, double* N2, cudaStream_t st) {
    DevInfo di;
    if (dev_info(&di) != 0) return cudaErrorUnknown;
    uint16_t* h = reinterpret_cast<uint16_t*>(s.perm_tmp);     // 2 m bytes of the 4 m there
    int64_t hb = (m + 8 * 256 - 1) / (8 * 256);
    if (hb > (int64_t)di.sms * 8) hb = (int64_t)di.sms * 8;
    k_hash16<<<(int)hb, 256, 0, st>>>(m, (uint32_t)d, seed, h);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool vec = (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (lda % 4 == 0) && (n % 4 == 0);
    // CTAs: one per SM (16 warps, 8 16-byte loads in flight per lane; two
    // 256-thread CTAs per SM measured slower), at least ceil(d /
    // kOwnMaxBuckets), at most d
    int64_t G = di.sms;
    const int64_t gmin = ((int64_t)d + kOwnMaxBuckets - 1) / kOwnMaxBuckets;
    if (G < gmin) G = gmin;
    if (G > d) G = d;
    static const int cap_env = env_int("CSK_SKETCH_OWN_CAP", 0);
    int64_t cap = (3 * (m / G) / 2 + 511) / 256 * 256;
    if (cap < 1024) cap = 1024;
    if (cap > kOwnMaxCap) cap = kOwnMaxCap;
    if (cap_env > 0) cap = cap_env;
    const size_t smem = (size_t)2 * cap * sizeof(int32_t);
    const int n4 = n / 4;
    // 8-byte loads when rows are 8-byte aligned but not 16 (n even, n % 4 = 2)
    const bool vec2 = !vec && (reinterpret_cast<uintptr_t>(A) % 8 == 0) && (lda % 2 == 0) &&
                      (n % 2 == 0);
    const int n2 = n / 2;
    const void* fn = vec ? (n4 <= 32 ? (const void*)k_sketch_own<4, 1>
                            : n4 <= 64 ? (const void*)k_sketch_own<4, 2> : (const void*)k_sketch_own<4, 4>)
                   : vec2 ? (n2 <= 32 ? (const void*)k_sketch_own<2, 1>
                             : n2 <= 64 ? (const void*)k_sketch_own<2, 2> : (const void*)k_sketch_own<2, 4>)
                         : (n <= 32 ? (const void*)k_sketch_own<1, 1> : (const void*)k_sketch_own<1, 4>);
    e = ensure_smem_attr(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kOwnThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = CSK_SKETCH_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int capi = (int)cap;
    void* args[] = {(void*)&A, (void*)&lda, (void*)&n, (void*)&m, (void*)&B, (void*)&ldb,
                    (void*)&nrhs, (void*)&h, (void*)&d, (void*)&seed, (void*)&capi, (void*)&At,
                    (void*)&Bt, (void*)&N2, (void*)&s.perm, (void*)&s.off};
    e = cudaLaunchKernelExC(&cfg, fn, args);
    note_launches(2);
    return e;
}
}  // namespace

cudaError_t launch_sketch(int dtype, const void* A, int64_t lda, int64_t m, int n, const void* B,
                          int64_t ldb, int nrhs, const SortScratch& s, int d, uint64_t seed,
                          void* At, void* Bt, double* N2, cudaStream_t st) {
    if (use_owner_path(dtype, A, lda, m, n, d, nrhs))
        return launch_sketch_own(static_cast<const float*>(A), lda, m, n,
                                 nrhs > 0 ? static_cast<const float*>(B) : nullptr, ldb, nrhs, s, d,
                                 seed, static_cast<float*>(At), static_cast<float*>(Bt), N2, st);
    cudaError_t e = launch_bucket_group(m, d, seed, s, st);
    if (e != cudaSuccess) return e;
    return launch_segsum(dtype, A, lda, m, n, nrhs > 0 ? B : nullptr, ldb, nrhs, s, d, seed, At, Bt,
                         N2, st);
}

cudaError_t launch_row_norms(int dtype, const void* A, int64_t ld, int rows, int n, double* N2,
                             cudaStream_t st) {
    DevInfo di;
    if (dev_info(&di) != 0) return cudaErrorUnknown;
    int64_t blocks = ((int64_t)rows + 8 * kNormRows - 1) / (8 * kNormRows);   // 8 warps per block
    if (blocks > (int64_t)di.sms * 32) blocks = (int64_t)di.sms * 32;
    if (dtype == CSK_F32)
        k_row_norms<float><<<(int)blocks, 256, 0, st>>>((const float*)A, ld, rows, n, N2);
    else
        k_row_norms<double><<<(int)blocks, 256, 0, st>>>((const double*)A, ld, rows, n, N2);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_norm2(int dtype, const void* v, int64_t len, double* out, cudaStream_t st) {
    if (dtype == CSK_F32)
        k_norm2<float><<<1, 1024, 0, st>>>((const float*)v, len, out);
    else
        k_norm2<double><<<1, 1024, 0, st>>>((const double*)v, len, out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace csk
