// gram.cu -- G = At At^T on the sm_103a tensor cores (tcgen05 + TMA + TMEM),
// in split BF16.
//
// The GRAM residual path updates r_{k+1} = r_k - alpha_k G[:, i_k], which
// follows from the projection of Algorithm 1 (r = bt - At x, so a step along
// At_{i_k}^T changes r by -alpha At At_{i_k}^T).  G is formed once:
//   hi = bf16(At), lo = bf16(At - hi)          (k_split_bf16)
//   G  ~= hi hi^T + hi lo^T + lo hi^T          (k_gram_tc, FP32 accumulation)
// The dropped lo lo^T term and the rounding of lo leave a relative error of
// about 2^-16 per product.  Only tiles on or above the diagonal are computed;
// each off-diagonal tile is also stored transposed, so G is exactly
// symmetric.  Finally G_jj := fl32(||At_j||^2) from the FP64 row norms
// (k_gram_diag), which makes the residual update of the chosen row consistent
// with the FP64 step length.
//
// k_gram_tc: persistent, one CTA per SM, 128 x 256 output tiles.
//   warp 0 / lane 0   TMA producer: 32-wide K chunks of hi and lo of the 128
//                     A-rows and of the 256 B-rows (four boxes, 48 KB) into a
//                     4-stage ring (64B swizzle)
//   warp 1 / lane 0   MMA issuer: tcgen05.mma kind::f16 (BF16 x BF16 -> FP32),
//                     M = 128, N = 256, K = 16; per stage the three products
//                     hi hi^T, hi lo^T, lo hi^T of both K halves (6 MMAs),
//                     into one of two TMEM accumulators (warp 1 allocates
//                     all 512 columns)
//   warps 2-5         epilogue: tcgen05.ld 32 lanes x 32 columns per warp;
//                     each 32 x 32 block wholly above the diagonal and
//                     inside G, and its transpose, are staged in shared
//                     memory (128B swizzle) and written by TMA tensor stores
//                     (one lane issues them); blocks on the diagonal or
//                     crossing column d use direct and mirrored per-lane
//                     stores (a tensor store clips at 16-byte granules, so
//                     a block crossing column d would write past it);
//                     the epilogue overlaps the next tile's MMAs
// Loading hi and lo of a chunk once for all three products moves 2/3 of the
// operand bytes per MMA that three (hi, hi), (hi, lo), (lo, hi) passes over
// K would, and a 48 KB stage holds 1.5x the MMA work of a (hi, hi) stage.
// Every mbarrier wait is bounded; on expiry the CTA records CSK_ETIMEOUT,
// drains its own TMA loads (bounded), frees its TMEM and returns.
#include <cstdlib>
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>

#include "async.cuh"
#include "common.cuh"
#include "kernels.h"

namespace csk {

namespace {

constexpr int BM = 128, BN = 256, BK = 32;
constexpr int KPAD = 64;                      // K padded to a multiple of 64 (the error bound's M)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;          // 8 KB per operand (hi or lo)
constexpr int B_BYTES = BN * BK * 2;          // 16 KB
// stage: [A hi | A lo | B hi | B lo]
constexpr int OFF_ALO = A_BYTES, OFF_BHI = 2 * A_BYTES, OFF_BLO = 2 * A_BYTES + B_BYTES;
constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);
// epilogue staging: per epilogue warp a 32 x 32 FP32 block and its transpose
constexpr int EPI_BLOCK = 32 * 32 * 4;                      // 4 KB
constexpr int EPI_BYTES = 4 * 2 * EPI_BLOCK;                // 32 KB
constexpr size_t kGramSmem = (size_t)STAGES * STAGE_BYTES + EPI_BYTES + 1024;
constexpr int TMEM_COLS = 2 * BN;             // two accumulators: MMA and epilogue overlap
constexpr int kGramThreads = 192;             // 6 warps: TMA, MMA, 4 x epilogue
constexpr uint32_t kWaitLimit = 1u << 26;     // try_wait polls before giving up

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------ PTX helpers
// (mbarrier helpers: async.cuh)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    return csk::mbar_wait(bar, parity, kWaitLimit);
}
// L2 policy for the BF16 operands: keep them resident (evict last).  The
// operands (d_pad x k_pad x 2 x 2 bytes, 82 MB at d = 20000, n = 1000) fit in
// the 129 MB L2, but the 1.6 GB of G written meanwhile would otherwise push
// them out, and a stage that misses L2 stalls the tensor pipe.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "l"(policy)
        : "memory");
}
// The same load multicast to the CTAs of `mask` in the cluster: the box lands
// at the same shared-memory offset in each and completes its bytes on the
// mbarrier at the same offset there.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                               int c0, int c1, uint16_t mask, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        ".multicast::cluster.L2::cache_hint [%0], [%1, {%3, %4}], [%2], %5, %6;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "h"(mask), "l"(policy)
        : "memory");
}
// L2 policy for G: written once here, read much later -- evict first, so
// the operands stay resident.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// Shared -> global tensor store of one box at (c0, c1), in this thread's
// bulk group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int c0, int c1,
                                             uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint"
        " [%0, {%2, %3}], [%1], %4;" ::"l"(reinterpret_cast<uint64_t>(map)), "r"(src), "r"(c0),
        "r"(c1), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// This thread's bulk groups have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// ... and have completed.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}
// Completion of this CTA's MMAs arrives on the mbarrier at the same offset in
// every CTA of `mask` (both CTAs of a pair release a stage they share).
__device__ __forceinline__ void tc_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(bar), "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, 64B swizzle,
// rows of 64 bytes (BK = 32 BF16), 8-row core groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused here)
    d |= (uint64_t)(512 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)4 << 61;                         // swizzle: 64B
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B, FP32 D,
// both K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4)                 // D format F32
                            | (1u << 7)               // A format BF16
                            | (1u << 10)              // B format BF16
                            | ((uint32_t)(BN >> 3) << 17)
                            | ((uint32_t)(BM >> 4) << 24);

// Tile order: row blocks are taken in groups of kGroupRows; inside a group the
// tiles run column block by column block, so the CTAs working at the same
// time share a few A panels and B panels in L2.  Only tiles with an element
// on or above the diagonal are enumerated, and CTA b takes the valid tiles
// b, b + grid, ... of that order, so no CTA holds more than
// ceil(valid / grid) of them.
//
// Pairs of CTAs take the same order with units of two row blocks (2p and
// 2p + 1, sharing the B panel of column block bj) in groups of
// kGroupRows / 2; a pair is valid when its upper row block is.
constexpr int kGroupRows = 8;     // row blocks per group of the tile order (8, 16, 32, 64 measured; 8 best)

// Position in the valid-unit order: group g, column block bj, and q, the
// index among the group's valid units of that column (the valid units of a
// column are the group's first ones, those whose top row is at most the
// column block's last column).
struct TileCursor {
    int g, bj, q;
    int nu, nbj, R, UH, ngroups;

    __host__ __device__ int count(int gg, int jj) const {
        const int lo = gg * R;
        int top = min(lo + R - 1, nu - 1);
        top = min(top, (jj * BN + BN - 1) / UH);
        return top >= lo ? top - lo + 1 : 0;
    }
    // first column block with a valid unit in group gg (at most nbj - 1:
    // the last column block reaches the last unit)
    __host__ __device__ int first_col(int gg) const {
        const int need = gg * R * UH - BN + 1;
        return need <= 0 ? 0 : (need + BN - 1) / BN;
    }
    // Moves k valid units on; false past the last one.
    __host__ __device__ bool advance(int k) {
        q += k;
        while (g < ngroups) {
            const int c = count(g, bj);
            if (q < c) return true;
            q -= c;
            if (++bj == nbj) {
                ++g;
                bj = g < ngroups ? first_col(g) : 0;
            }
        }
        return false;
    }
    __host__ __device__ int unit() const { return g * R + q; }
};

// Cursor at valid unit `first` (false if there are fewer units).
template <bool PAIR>
__host__ __device__ __forceinline__ bool tile_cursor(int nbi, int nbj, int first, TileCursor* c) {
    c->nu = PAIR ? nbi / 2 : nbi;
    c->R = PAIR ? kGroupRows / 2 : kGroupRows;
    c->UH = PAIR ? 2 * BM : BM;
    c->nbj = nbj;
    c->ngroups = (c->nu + c->R - 1) / c->R;
    c->g = 0;
    c->bj = 0;
    c->q = 0;
    return c->advance(first);
}

// ----------------------------------------------------------------- kernels
// Each thread converts 8 consecutive columns of a row (k_pad is a multiple
// of 64, so a chunk never crosses a row): two 16-byte loads of At when the
// row segment is aligned and inside [0, n), one 16-byte store into hi and
// one into lo.  Padding rows and columns are written as zeros.
__global__ void k_split_bf16(const float* __restrict__ At, int d, int n, int d_pad, int k_pad,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const int kc = k_pad / 8;                               // chunks per row
    const int64_t total = (int64_t)d_pad * kc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t sq = stride / kc;
    const int sr = (int)(stride - sq * kc);
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t r = e / kc;
    int c = (int)(e - r * kc);
    const bool vec = (n % 4 == 0) && (reinterpret_cast<uintptr_t>(At) % 16 == 0);
    for (; e < total; e += stride) {
        float a[8];
        const int c0 = c * 8;
        const float* src = At + r * (int64_t)n + c0;
        if (r < d && vec && c0 + 8 <= n) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(src));
            const float4 v = __ldg(reinterpret_cast<const float4*>(src) + 1);
            a[0] = u.x; a[1] = u.y; a[2] = u.z; a[3] = u.w;
            a[4] = v.x; a[5] = v.y; a[6] = v.z; a[7] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = (r < d && c0 + q < n) ? __ldg(src + q) : 0.0f;
        }
        uint32_t h2[4], l2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(a[2 * q]);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(a[2 * q + 1]);
            // a - h is exact in FP32
            const __nv_bfloat16 e0 = __float2bfloat16_rn(a[2 * q] - __bfloat162float(h0));
            const __nv_bfloat16 e1 = __float2bfloat16_rn(a[2 * q + 1] - __bfloat162float(h1));
            h2[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            l2[q] = (uint32_t)__bfloat16_as_ushort(e0) | ((uint32_t)__bfloat16_as_ushort(e1) << 16);
        }
        reinterpret_cast<uint4*>(hi)[e] = make_uint4(h2[0], h2[1], h2[2], h2[3]);
        reinterpret_cast<uint4*>(lo)[e] = make_uint4(l2[0], l2[1], l2[2], l2[3]);
        r += sq;
        c += sr;
        if (c >= kc) { c -= kc; ++r; }
    }
}

// Persistent: CTA b computes tiles b, b + grid, ...  Warp 0 / lane 0 loads
// K chunks through a 4-stage TMA ring; warp 1 / lane 0 issues the MMAs into
// one of two TMEM accumulators; warps 2-5 drain the other accumulator to
// global memory, so a tile's epilogue overlaps the next tile's MMAs.
// Element (r, c) is written, with its mirror (c, r), exactly when c >= r.
//
// PAIR: launched in clusters of two CTAs that take the tiles (2p, bj) and
// (2p + 1, bj) together.  Each loads its own A panels (hi, lo) and half of
// the shared B panels (128 of their 256 rows), multicast into both CTAs'
// stage, so a stage costs each SM 32 KB of L2 reads instead of 48 KB; each
// CTA's stage barrier expects all 48 KB, and a stage is refilled only after both CTAs' MMAs
// released it (their commits arrive on both CTAs' empty barriers, count 2).
// Cluster barriers after set-up and before exit keep each CTA resident while
// its peer may still write into its shared memory.
template <bool PAIR>
__global__ void __launch_bounds__(kGramThreads, 1)
k_gram_tc(const __grid_constant__ CUtensorMap map_hi_a, const __grid_constant__ CUtensorMap map_lo_a,
          const __grid_constant__ CUtensorMap map_hi_b, const __grid_constant__ CUtensorMap map_lo_b,
          const __grid_constant__ CUtensorMap map_g, int g_tma,
          int d, int kchunks, int nbi, int nbj, float* __restrict__ G, int64_t ldg,
          csk_info* info) {
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(smem_u32(&full_bar[st]), 1);
            mbar_init(smem_u32(&empty_bar[st]), PAIR ? 2 : 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&acc_full[a]), 1);
            mbar_init(smem_u32(&acc_empty[a]), 4);      // one arrival per epilogue warp
        }
        fail_sh = 0;
        mbar_fence_init();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (PAIR) cluster_sync_all();          // both CTAs' barriers exist before any load
    const uint32_t tmem = tmem_base_sh;
    const int nch = kchunks;
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
    const int first = PAIR ? (int)blockIdx.x / 2 : (int)blockIdx.x;
    const int step = PAIR ? (int)gridDim.x / 2 : (int)gridDim.x;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            const uint64_t pol = l2_evict_last_policy();
            int64_t g = 0;                 // chunk counter over all tiles of this CTA
            int64_t issued = 0;
            bool ok = true;
            TileCursor cur;
            for (bool more = tile_cursor<PAIR>(nbi, nbj, first, &cur); more && ok;
                 more = cur.advance(step)) {
                const int bi = PAIR ? 2 * cur.unit() + (int)rank : cur.unit(), bj = cur.bj;
                for (int c = 0; c < nch; ++c, ++g) {
                    const int st = (int)(g % STAGES);
                    const int64_t r = g / STAGES;
                    if (r > 0 && !mbar_wait(smem_u32(&empty_bar[st]), (uint32_t)((r - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    const int kx = c * BK;
                    const uint32_t sa = smem_u32(dsm + st * STAGE_BYTES);
                    const uint32_t fb = smem_u32(&full_bar[st]);
                    mbar_expect_tx(fb, STAGE_BYTES);
                    tma_load_2d(sa, &map_hi_a, fb, kx, bi * BM, pol);
                    tma_load_2d(sa + OFF_ALO, &map_lo_a, fb, kx, bi * BM, pol);
                    if (PAIR) {
                        const uint32_t half = rank * (B_BYTES / 2);
                        const int brow = bj * BN + (int)rank * BM;
                        tma_load_2d_mc(sa + OFF_BHI + half, &map_hi_a, fb, kx, brow, (uint16_t)3, pol);
                        tma_load_2d_mc(sa + OFF_BLO + half, &map_lo_a, fb, kx, brow, (uint16_t)3, pol);
                    } else {
                        tma_load_2d(sa + OFF_BHI, &map_hi_b, fb, kx, bj * BN, pol);
                        tma_load_2d(sa + OFF_BLO, &map_lo_b, fb, kx, bj * BN, pol);
                    }
                    issued = g + 1;
                }
            }
            if (!ok) {
                atomicExch(&fail_sh, 1);
                for (int64_t q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q)
                    (void)mbar_wait(smem_u32(&full_bar[q % STAGES]), (uint32_t)((q / STAGES) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            int64_t g = 0;
            int tc = 0;
            bool ok = true;
            TileCursor cur;
            for (bool more = tile_cursor<PAIR>(nbi, nbj, first, &cur); more && ok;
                 more = cur.advance(step)) {
                const int a = tc & 1, u = tc >> 1;
                ++tc;
                if (u > 0 && !mbar_wait(smem_u32(&acc_empty[a]), (uint32_t)((u - 1) & 1))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(a * BN);
                for (int c = 0; c < nch; ++c, ++g) {
                    const int st = (int)(g % STAGES);
                    if (!mbar_wait(smem_u32(&full_bar[st]), (uint32_t)((g / STAGES) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(dsm + st * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t ah = smem_desc_sw64(sa + kk * 32);
                        const uint64_t al = smem_desc_sw64(sa + OFF_ALO + kk * 32);
                        const uint64_t bh = smem_desc_sw64(sa + OFF_BHI + kk * 32);
                        const uint64_t bl = smem_desc_sw64(sa + OFF_BLO + kk * 32);
                        tc_mma_bf16(dt, ah, bh, kIdesc, (c > 0 || kk > 0) ? 1u : 0u);
                        tc_mma_bf16(dt, ah, bl, kIdesc, 1u);
                        tc_mma_bf16(dt, al, bh, kIdesc, 1u);
                    }
                    if (PAIR) tc_commit_mc(smem_u32(&empty_bar[st]), (uint16_t)3);
                    else tc_commit(smem_u32(&empty_bar[st]));
                }
                if (ok) tc_commit(smem_u32(&acc_full[a]));
            }
            if (!ok) atomicExch(&fail_sh, 1);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 * (w % 4) .. + 31
        const int quad = warp & 3;
        const bool vec_ok = (ldg % 4 == 0) && (reinterpret_cast<uintptr_t>(G) % 16 == 0);
        // staging of this warp: [block | transpose], 1024-byte aligned (128B swizzle)
        const uint32_t stg = smem_u32(dsm + STAGES * STAGE_BYTES) + (uint32_t)(quad * 2 * EPI_BLOCK);
        const uint32_t stg_t = stg + EPI_BLOCK;
        const uint64_t gpol = l2_evict_first_policy();
        int tc = 0;
        TileCursor cur;
        for (bool more = tile_cursor<PAIR>(nbi, nbj, first, &cur); more; more = cur.advance(step)) {
            const int bi = PAIR ? 2 * cur.unit() + (int)rank : cur.unit(), bj = cur.bj;
            const int a = tc & 1, u = tc >> 1;
            ++tc;
            const bool ok = mbar_wait(smem_u32(&acc_full[a]), (uint32_t)(u & 1));
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicExch(&fail_sh, 1);
                break;
            }
            tc_fence_after();
            const int row0 = bi * BM + quad * 32;
            const int row = row0 + lane;
            const bool upper = (bj * BN) >= (bi * BM + BM);     // every column > every row
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * BN + c0), v);
                const int col0 = bj * BN + c0;
                // 32 x 32 blocks wholly above the diagonal and inside G go
                // through the tensor stores (also on the diagonal band tiles)
                if (g_tma && col0 >= row0 + 32 && row0 + 32 <= d && col0 + 32 <= d) {
                    // the staging buffers are free once the previous stores read them
                    if (lane == 0) bulk_wait_read_all();
                    __syncwarp();
                    // block: row `lane`, 16-byte chunk j at position j ^ (lane % 8)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t dst = stg + (uint32_t)(lane * 128 + ((j ^ (lane & 7)) << 4));
                        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst),
                                     "r"(v[4 * j]), "r"(v[4 * j + 1]), "r"(v[4 * j + 2]),
                                     "r"(v[4 * j + 3])
                                     : "memory");
                    }
                    // transpose: row q (column col0 + q of G), element `lane`
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const uint32_t dst = stg_t + (uint32_t)(q * 128 +
                                                                (((lane >> 2) ^ (q & 7)) << 4) +
                                                                ((lane & 3) << 2));
                        asm volatile("st.shared.b32 [%0], %1;" ::"r"(dst), "r"(v[q]) : "memory");
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&map_g, stg, col0, row0, gpol);      // G[row0.., col0..]
                        tma_store_2d(&map_g, stg_t, row0, col0, gpol);    // G[col0.., row0..]
                        bulk_commit();
                    }
                } else if (upper) {
                    if (row < d) {
                        float* dst = G + (int64_t)row * ldg + col0;
                        // streaming stores: G is written once here and read much
                        // later, so keep the BF16 operands resident in L2 instead
                        if (vec_ok && col0 + 32 <= d) {
#pragma unroll
                            for (int q = 0; q < 32; q += 4)
                                __stcs(reinterpret_cast<float4*>(dst + q),
                                       make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                                   __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3])));
                        } else {
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                if (col0 + q < d) __stcs(dst + q, __uint_as_float(v[q]));
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (col0 + q < d && row < d)
                            __stcs(G + (int64_t)(col0 + q) * ldg + row, __uint_as_float(v[q]));
                } else if (col0 + 32 > row0) {
                    // block on the diagonal: (r, c) and (c, r) are summed in
                    // different orders, so keep c >= r and mirror it (blocks
                    // wholly below the diagonal are their mirrors' images)
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int col = col0 + q;
                        if (row < d && col < d && col >= row) {
                            __stcs(G + (int64_t)row * ldg + col, __uint_as_float(v[q]));
                            __stcs(G + (int64_t)col * ldg + row, __uint_as_float(v[q]));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty[a]));
        }
        // every tensor store of this warp has completed before the CTA exits
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && fail_sh && info) set_status_once(info, CSK_ETIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
    if (PAIR) cluster_sync_all();          // the peer no longer writes into this CTA
}

__global__ void k_gram_diag(const double* __restrict__ N2, int d, float* __restrict__ G, int64_t ldg) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
        G[(int64_t)j * ldg + j] = (float)N2[j];
}

// --------------------------------------------------------------- host side
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_map(CUtensorMap* map, void* base, int rows, int cols, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// G (d x d FP32, row stride ldg) as 32 x 32 boxes with 128B swizzle, for the
// epilogue's tensor stores; false when G's base or row stride is not a
// multiple of 16 bytes (the per-lane stores are used then).
bool make_g_map(CUtensorMap* map, float* G, int d, int64_t ldg) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || reinterpret_cast<uintptr_t>(G) % 16 != 0 || (ldg * 4) % 16 != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)d};
    const cuuint64_t strides[1] = {(cuuint64_t)ldg * 4};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, G, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Pairs of CTAs sharing B panels (the default); CSK_GRAM_PAIR=0 in the
// environment selects the one-CTA kernel (same products, same bits), for
// comparisons.
bool gram_pairs_enabled() {
    static const bool on = [] {
        const char* v = getenv("CSK_GRAM_PAIR");
        return !(v && v[0] == '0');
    }();
    return on;
}

}  // namespace

int64_t gram_ld(int d) { return round_up(d, 32); }

size_t gram_scratch_bytes(int d, int n) {
    const int64_t dp = round_up(d, BN), kp = round_up(n, KPAD);
    return (size_t)(2 * dp * kp * 2 + 1024);
}

cudaError_t launch_gram_split_bf16(const float* At, int d, int n, const double* N2, float* G,
                                   int64_t ldg, void* scratch, csk_info* info, cudaStream_t st) {
    const int dp = (int)round_up(d, BN), kp = (int)round_up(n, KPAD);
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(scratch) + 1023) & ~uintptr_t(1023));
    __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* lo = hi + (size_t)dp * kp;
    DevInfo di;
    if (dev_info(&di) != 0) return cudaErrorUnknown;
    k_split_bf16<<<di.sms * 8, 256, 0, st>>>(At, d, n, dp, kp, hi, lo);
    CUtensorMap mha, mla, mhb, mlb;
    if (!make_map(&mha, hi, dp, kp, BM) || !make_map(&mla, lo, dp, kp, BM) ||
        !make_map(&mhb, hi, dp, kp, BN) || !make_map(&mlb, lo, dp, kp, BN))
        return cudaErrorInvalidValue;
    CUtensorMap mg;
    memset(&mg, 0, sizeof(mg));
    const int g_tma = make_g_map(&mg, G, d, ldg) ? 1 : 0;
    const size_t smem = kGramSmem;
    const int nbi = dp / BM, nbj = dp / BN;          // nbi is even (dp is a multiple of BN)
    cudaError_t e;
    if (gram_pairs_enabled()) {
        e = ensure_smem_attr((const void*)k_gram_tc<true>, smem);
        if (e != cudaSuccess) return e;
        const int npairs = nbi / 2;
        int valid = 0;
        for (int q = 0; q < npairs; ++q) valid += nbj - q;
        const int pairs = valid < di.sms / 2 ? valid : di.sms / 2;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * pairs));
        cfg.blockDim = dim3(kGramThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, k_gram_tc<true>, mha, mla, mhb, mlb, mg, g_tma, d, kp / BK,
                               nbi, nbj, G, ldg, info);
        if (e != cudaSuccess) return e;
    } else {
        e = ensure_smem_attr((const void*)k_gram_tc<false>, smem);
        if (e != cudaSuccess) return e;
        int valid = 0;
        for (int i = 0; i < nbi; ++i) valid += nbj - (i * BM) / BN;
        const int grid = valid < di.sms ? valid : di.sms;
        k_gram_tc<false><<<grid, kGramThreads, smem, st>>>(mha, mla, mhb, mlb, mg, g_tma, d,
                                                           kp / BK, nbi, nbj, G, ldg, info);
    }
    if (N2) k_gram_diag<<<(d + 255) / 256, 256, 0, st>>>(N2, d, G, ldg);
    note_launches(N2 ? 3 : 2);
    return cudaGetLastError();
}

}  // namespace csk
