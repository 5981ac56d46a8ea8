// batched.cu -- many independent CSK solves (systems of uneven m, n, d, each
// with many right-hand sides) in one persistent launch.
//
// Per system s the stream carries its sketch (At_s = S_s A_s, Bt_s = S_s B_s,
// FP64 row norms) and its split-BF16 Gram matrix G_s = At_s At_s^T (the same
// kernels as csk_sketch / csk_gram).  Then one persistent kernel runs every
// (system, right-hand side) pair -- a "unit" -- to completion: a CTA takes the
// next unit from an atomic counter (units are ordered by decreasing d*n so the
// long solves start first) and runs the whole MWRK loop of Algorithm 1 on it
// alone, with r, the row weights and x in its shared memory and the GRAM
// residual update r -= alpha G_s[i_k, :] (r_{i_k} = 0 exactly).  A step costs
// one pass over the CTA's rows and one CTA barrier; no CTA waits for another.
// The final check (FP64 RES; ||bt - At x|| / ||bt|| with a compensated FP32
// dot product, GB300's FP64 rate being a small fraction of FP32) is done by
// the same CTA.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <utility>
#include <vector>

#include "async.cuh"
#include "common.cuh"
#include "fp64.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace csk {

namespace {

// State of one (system, right-hand side) unit between calls that run it a
// step budget at a time (32 bytes, zero = not started).
struct UnitState {
    int64_t k;            // steps done
    int32_t idx;          // the pending projection's row (applied at the next pass), -1 none
    float alpha;          //   and its step length
    float threshold;      // tol * ||x*||^2 (or tol * ||bt||^2)
    int32_t started;      // 1 once the unit has run
    int32_t done;         // 1 once it has finished (outputs and info written)
    int32_t pad_;
};

struct BatchSys {
    const float* At;
    const float* Bt;
    const double* N2;
    const float* G;
    const float* X0;
    const float* Xstar;
    float* Xout;
    csk_info* info;
    UnitState* states;    // nrhs
    float* rst;           // nrhs x d: residuals of suspended units
    float* xst;           // nrhs x n: iterates of suspended units
    int64_t ldg;
    int32_t d, n, nrhs, unit_begin;
};

constexpr int kTableChunk = 32;   // descriptors per table-writing launch (params < 4 KB)

struct TableChunk {
    BatchSys e[kTableChunk];
    int count, first;
};

__global__ void k_write_table(TableChunk c, BatchSys* table) {
    const int i = threadIdx.x;
    if (i < c.count) table[c.first + i] = c.e[i];
}

constexpr int kMaxWarps = 32;

struct BatchShared {
    RedShared<float, kMaxWarps> red;
    double dbuf[kMaxWarps];
    uint64_t gbar;          // completion of the bulk copy of a G row's head
    int unit;
    int fail;               // a staging wait ran out: this CTA stops
};

constexpr uint32_t kStageWait = 1u << 26;   // try_wait polls for a staged row head

__device__ __forceinline__ double block_sum_f64(double v, BatchShared& sh) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh.dbuf[warp] = v;
    __syncthreads();
    double s = lane < nw ? sh.dbuf[lane] : 0.0;
    return warp_sum(s);
}

// Error-free sum of two floats (Knuth's TwoSum): s + t == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = a + b;
    const float bb = s - a;
    t = (a - (s - bb)) + (b - bb);
}

constexpr int kGChunk = 8;     // G-row values per thread per chunk (two groups of four; two chunks in flight)
constexpr int kXChunk = 4;     // At-row values per thread in flight at once
constexpr int kRefreshRows = 4;   // rows a warp sums at once in the FP64 refresh

// Monotone code of a selection key: NaN highest (a numerical failure must
// reach the decision), "no candidate" (a zero row) lowest, otherwise the
// key's bits + 1 (keys are >= 0).  Larger code wins; equal codes -> smaller
// row, the ordering of better().
__device__ __forceinline__ uint32_t key_code(float key) {
    return key != key ? 0xFFFFFFFFu : __float_as_uint(key) + 1u;
}

// Logs of one unit (ik / x NULL for every other unit): i_k of step k and x_k,
// the iterate step k selects from (n floats per step).
struct UnitLog {
    int32_t* ik;  int64_t ik_len;
    float* x;     int64_t x_len;
};

// One unit, resumed from its state when it has run before; with budget > 0
// it stops after `budget` more steps, saves r, x and the pending projection
// in its state and reports CSK_INPROGRESS (no outputs yet).
//
// G[i_k, 0..H) (H = the launch's staging capacity, a multiple of 4 times the
// CTA's threads, or the whole row when it fits) arrives in shared memory by
// one bulk copy per step, issued by thread 0 and completed on sh.gbar; the
// rest of the row streams through registers, its first chunk loaded while
// the copy is in flight.  Thread tid scores the groups of four rows g = tid
// (mod threads) in increasing order either way, so the results do not
// depend on H.
__device__ __forceinline__ void solve_unit(const BatchSys& S, int rhs, float* sm, BatchShared& sh, float tol,
                           int64_t max_iter, int refresh, const UnitLog& lg, int64_t budget,
                           int H, uint32_t& gphase) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    const int d = S.d, n = S.n, R = S.nrhs;
    const int dpad = (d + 3) & ~3, npad = (n + 3) & ~3;
    float* rs = sm;
    float* w2s = rs + dpad;
    float* xs = w2s + dpad;
    float* xss = xs + npad;
    float* gs = xss + npad;                   // staged head of G[idx, :] (16-byte aligned)
    int par = 0;
    UnitState* ust = S.states + rhs;
    if (ust->done) return;                    // finished in an earlier call
    const bool resume = ust->started != 0;
    float* rsave = S.rst + (int64_t)rhs * d;
    float* xsave = S.xst + (int64_t)rhs * n;

    for (int j = tid; j < d; j += nt) {
        rs[j] = resume ? rsave[j] : S.Bt[(int64_t)j * R + rhs];
        const double N = S.N2[j];
        w2s[j] = N > 0.0 ? (float)(1.0 / N) : (N == 0.0 ? -1.0f : NAN);
    }
    for (int c = tid; c < n; c += nt) {
        xs[c] = resume ? xsave[c] : (S.X0 ? S.X0[(int64_t)c * R + rhs] : 0.0f);
        xss[c] = S.Xstar ? S.Xstar[(int64_t)c * R + rhs] : 0.0f;
    }
    __syncthreads();
    // stopping threshold tol * ||x*||^2 (or tol * ||bt||^2 without x*)
    float threshold;
    if (resume) {
        threshold = ust->threshold;
    } else {
        double nrm = 0.0;
        if (S.Xstar) for (int c = tid; c < n; c += nt) nrm += (double)xss[c] * (double)xss[c];
        else for (int j = tid; j < d; j += nt) nrm += (double)rs[j] * (double)rs[j];
        nrm = block_sum_f64(nrm, sh);
        threshold = stop_threshold<float>(tol, nrm, S.Xstar ? n : d);
    }
    const bool fresh_r = (S.X0 != nullptr);
    const bool xstar = (S.Xstar != nullptr);
    int64_t k = resume ? ust->k : 0;
    int status = CSK_OK;
    int32_t idx = resume ? ust->idx : -1;
    float alpha = resume ? ust->alpha : 0.0f;
    const int64_t kend = budget > 0 ? k + budget : INT64_MAX;
    // next step at a multiple of `refresh` (one division per unit, none per step)
    int64_t next_refresh = refresh > 0 ? (k + refresh - 1) / refresh * refresh : (k == 0 ? 0 : -1);
    bool suspended = false;
    __syncthreads();                          // every thread has read the state
    for (;;) {
        const bool at_refresh = k == next_refresh;
        if (at_refresh && refresh > 0) next_refresh += refresh;
        if (k == 0 ? fresh_r : at_refresh) {
            // r = bt - At x with FP64 accumulation (x0 given, or periodic refresh)
            if (idx >= 0) {
                const float* arow = S.At + (int64_t)idx * n;
                for (int c = tid; c < n; c += nt) xs[c] = fmaf(alpha, arow[c], xs[c]);
                idx = -1;
            }
            __syncthreads();
            for (int j0 = warp * kRefreshRows; j0 < d; j0 += nw * kRefreshRows) {
                const int m = min(kRefreshRows, d - j0);
                const double acc = warp_rows_dot_f64<kRefreshRows>(S.At + (int64_t)j0 * n, n, m, xs, n, lane);
                const int u = transpose_row<kRefreshRows>(lane);
                if (transpose_rep<kRefreshRows>(lane) && u < m)
                    rs[j0 + u] = (float)(widen(S.Bt[(int64_t)(j0 + u) * R + rhs]) - acc);
            }
            __syncthreads();
        }
        // one pass: apply the previous step's update, then score.  Each
        // thread walks rows tid, tid + nt, ... as before, but issues the
        // loads of a whole chunk of G[idx, :] (and of its part of At[idx, :])
        // before using any, so a step waits for one memory round trip, not
        // one per row.
        Red<float> c;
        c.key = -1.0f; c.alpha = 0.0f; c.stat = 0.0f; c.idx = INT_MAX;
        const float* grow = idx >= 0 ? S.G + (int64_t)idx * S.ldg : nullptr;
        const float* arow = idx >= 0 ? S.At + (int64_t)idx * n : nullptr;
        float av[kXChunk];
#pragma unroll
        for (int q = 0; q < kXChunk; ++q) {
            const int col = tid + q * nt;
            av[q] = (arow && col < n) ? __ldg(arow + col) : 0.0f;
        }
        // Rows come in groups of four consecutive ones: thread tid takes the
        // groups tid, tid + nt, ... in increasing order (one 16-byte shared-
        // memory access per array per group), and row 4g + e goes to running
        // maximum e (a strict > keeps the first of equal codes), merged below:
        // the same winner as one sequential scan.
        uint32_t bc[4] = {0u, 0u, 0u, 0u};
        int32_t bi[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
        float ba[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const int ng = (d + 3) >> 2;           // row groups (the last may be partial)
        float4* rs4 = reinterpret_cast<float4*>(rs);
        const float4* w4s = reinterpret_cast<const float4*>(w2s);
        // one group: r -= alpha G[idx, rows] (r_idx = 0 exactly), scored
        auto group = [&](int g, float4 gg, bool upd) {
            const int j0 = 4 * g;
            float4 r4 = rs4[g];
            const float4 w4 = w4s[g];
            float rr[4] = {r4.x, r4.y, r4.z, r4.w};
            const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
            const float gx[4] = {gg.x, gg.y, gg.z, gg.w};
            const int nv = min(4, d - j0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (e < nv) {
                    float r = rr[e];
                    if (upd) r = (j0 + e == idx) ? 0.0f : fmaf(-alpha, gx[e], r);
                    rr[e] = r;
                    const float w = ww[e];
                    const uint32_t code = (w < 0.0f) ? 0u : key_code(r * r * w);
                    if (code > bc[e]) { bc[e] = code; bi[e] = j0 + e; ba[e] = r * w; }
                    if (!xstar) c.stat += r * r;
                }
            }
            if (upd) {
                if (nv == 4) rs4[g] = make_float4(rr[0], rr[1], rr[2], rr[3]);
                else
                    for (int e = 0; e < nv; ++e) rs[j0 + e] = rr[e];
            }
        };
        // the head of G[idx, :] by one bulk copy into shared memory
        const int hg = grow ? min(ng, H >> 2) : 0;      // staged groups
        if (hg > 0 && tid == 0) {
            const uint32_t bytes = (uint32_t)hg * 16u;
            mbar_expect_tx(smem_u32(&sh.gbar), bytes);
            bulk_g2s(smem_u32(gs), grow, bytes, smem_u32(&sh.gbar));
        }
        // the rest of G[idx, :] in chunks of kGChunk / 4 groups per thread,
        // the next chunk's loads issued before the current chunk is scored
        // (the first chunk's while the head is in flight)
        constexpr int KG = kGChunk / 4;
        const float4* grow4 = reinterpret_cast<const float4*>(grow);
        float4 gv[KG];
#pragma unroll
        for (int q = 0; q < KG; ++q) {
            const int g = hg + q * nt + tid;
            gv[q] = (grow && g < ng) ? __ldg(grow4 + g) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // x += alpha At[idx, :] and ||x - x*||^2 (nothing here reads G): done
        // while the head of the G row is in flight
        for (int base = 0; base < n; base += kXChunk * nt) {
#pragma unroll
            for (int q = 0; q < kXChunk; ++q) {
                const int col = base + q * nt + tid;
                if (col < n) {
                    float x = xs[col];
                    if (arow) {
                        x = fmaf(alpha, base == 0 ? av[q] : __ldg(arow + col), x);
                        xs[col] = x;
                    }
                    if (S.Xstar) {
                        const float t = x - xss[col];
                        c.stat += t * t;
                    }
                }
            }
        }
        if (hg > 0) {
            const bool ok = mbar_wait(smem_u32(&sh.gbar), gphase & 1u, kStageWait);
            ++gphase;
            if (!ok) sh.fail = 1;             // seen by all after the reduction's barrier
            const float4* gs4 = reinterpret_cast<const float4*>(gs);
            for (int g = tid; g < hg; g += nt) group(g, gs4[g], true);
        }
        for (int base = hg; base < ng; base += KG * nt) {
            float4 gn[KG];
            const int nb = base + KG * nt;
#pragma unroll
            for (int q = 0; q < KG; ++q) {
                const int g = nb + q * nt + tid;
                gn[q] = (grow && g < ng) ? __ldg(grow4 + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < KG; ++q) {
                const int g = base + q * nt + tid;
                if (g < ng) group(g, gv[q], grow != nullptr);
            }
#pragma unroll
            for (int q = 0; q < KG; ++q) gv[q] = gn[q];
        }
#pragma unroll
        for (int a = 1; a < 4; ++a)
            if (bc[a] > bc[0] || (bc[a] == bc[0] && bi[a] < bi[0])) {
                bc[0] = bc[a]; bi[0] = bi[a]; ba[0] = ba[a];
            }
        if (bc[0] != 0u) {
            c.key = bc[0] == 0xFFFFFFFFu ? NAN : __uint_as_float(bc[0] - 1u);
            c.alpha = ba[0];
            c.idx = bi[0];
        }
        c = block_reduce(c, sh.red, par);
        if (sh.fail) { status = CSK_ETIMEOUT; break; }
        if (c.stat <= threshold) { status = CSK_OK; break; }
        if (k >= max_iter) { status = CSK_MAXITER; break; }
        if (c.key != c.key || c.key < 0.0f) { status = CSK_ENUMERIC; break; }
        if (c.key == 0.0f) { status = CSK_OK; break; }
        // xs holds x_k here (the pass applied the previous step's update)
        if (lg.ik && k < lg.ik_len && tid == 0) lg.ik[k] = c.idx;
        if (lg.x && k < lg.x_len)
            for (int col = tid; col < n; col += nt) lg.x[k * n + col] = xs[col];
        idx = c.idx;
        alpha = c.alpha;
        ++k;
        if (k >= kend) { suspended = true; break; }
    }
    __syncthreads();
    if (suspended) {
        // r and x as of the last pass; the pending projection (idx, alpha)
        // is applied by the next call's first pass
        for (int j = tid; j < d; j += nt) rsave[j] = rs[j];
        for (int c = tid; c < n; c += nt) xsave[c] = xs[c];
        if (tid == 0) {
            ust->k = k;
            ust->idx = idx;
            ust->alpha = alpha;
            ust->threshold = threshold;
            ust->started = 1;
            csk_info* info = S.info + rhs;
            info->status = CSK_INPROGRESS;
            info->path = CSK_RESID_GRAM;
            info->iters = k;
            info->rse = (double)NAN;
            info->resid = (double)NAN;
            info->rows = d;
            info->grid = (int32_t)gridDim.x;
        }
        __syncthreads();
        return;
    }
    // outputs and final check
    for (int col = tid; col < n; col += nt) S.Xout[(int64_t)col * R + rhs] = xs[col];
    double ee = 0.0, ss = 0.0;
    if (S.Xstar)
        for (int col = tid; col < n; col += nt) {
            const double e = (double)xs[col] - (double)xss[col];
            ee += e * e;
            ss += (double)xss[col] * (double)xss[col];
        }
    double rr = 0.0, bb = 0.0, empty = 0.0;
    for (int j = tid; j < d; j += nt) empty += (w2s[j] < 0.0f) ? 1.0 : 0.0;
    for (int j = warp; j < d; j += nw) {
        const float* a = S.At + (int64_t)j * n;
        float hi = 0.0f, lo = 0.0f;
        for (int col = lane; col < n; col += 32) {
            const float p = a[col] * xs[col];
            const float e = fmaf(a[col], xs[col], -p);
            float s, t;
            two_sum(hi, p, s, t);
            hi = s;
            lo += t + e;
        }
        double dot = (double)hi + (double)lo;
        dot = warp_sum(dot);
        if (lane == 0) {
            const double bj = (double)S.Bt[(int64_t)j * R + rhs];
            const double r = bj - dot;
            rr += r * r;
            bb += bj * bj;
        }
    }
    ee = block_sum_f64(ee, sh);
    ss = block_sum_f64(ss, sh);
    rr = block_sum_f64(rr, sh);
    bb = block_sum_f64(bb, sh);
    empty = block_sum_f64(empty, sh);
    if (tid == 0) {
        ust->done = 1;
        ust->k = k;
        csk_info* info = S.info + rhs;
        info->status = status;
        info->path = CSK_RESID_GRAM;
        info->iters = k;
        info->rse = S.Xstar ? ee / ss : (double)NAN;
        info->resid = sqrt(rr / bb);
        info->rows = d;
        info->empty_rows = (int32_t)empty;
        info->grid = (int32_t)gridDim.x;
        info->reserved0 = 0;
        info->reserved1 = 0.0;
        info->reserved2 = 0.0;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(512)
k_iterate_batched(const BatchSys* __restrict__ table, int nsys, int nunits, int* counter, float tol,
                  int64_t max_iter, int refresh, int log_unit, UnitLog lg, int64_t budget, int H) {
    extern __shared__ __align__(16) float sm[];
    __shared__ BatchShared sh;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&sh.gbar), 1);
        mbar_fence_init();
        sh.fail = 0;
    }
    __syncthreads();
    uint32_t gphase = 0;                       // bulk copies completed on sh.gbar
    for (;;) {
        if (threadIdx.x == 0) sh.unit = sh.fail ? nunits : atomicAdd(counter, 1);
        __syncthreads();
        const int u = sh.unit;
        __syncthreads();
        if (u >= nunits) break;
        // system of unit u: last s with unit_begin <= u (table ordered by unit_begin)
        int lo = 0, hi = nsys - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (table[mid].unit_begin <= u) lo = mid; else hi = mid - 1;
        }
        const BatchSys S = table[lo];
        const UnitLog none = {nullptr, 0, nullptr, 0};
        solve_unit(S, u - S.unit_begin, sm, sh, tol, max_iter, refresh, u == log_unit ? lg : none,
                   budget, H, gphase);
    }
    // a copy whose wait ran out may still be writing this CTA's shared memory
    if (sh.fail && threadIdx.x == 0)
        (void)mbar_wait(smem_u32(&sh.gbar), (gphase - 1u) & 1u, kStageWait);
}

inline size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

// A system's resident area: its sketch, Gram matrix and unit states, kept on
// the device between the calls that iterate it (serving keeps it from the
// request's arrival to its retirement).
struct AreaLayout {
    size_t At, Bt, N2, G, states, rst, xst, total;
};

void area_layout(int64_t n, int64_t d, int32_t nrhs, AreaLayout* A) {
    size_t o = 0;
    A->At = o;     o += a256((size_t)d * n * 4);
    A->Bt = o;     o += a256((size_t)d * nrhs * 4);
    A->N2 = o;     o += a256((size_t)d * 8);
    A->G = o;      o += a256((size_t)d * gram_ld((int)d) * 4);
    A->states = o; o += a256((size_t)nrhs * sizeof(UnitState));
    A->rst = o;    o += a256((size_t)nrhs * d * 4);
    A->xst = o;    o += a256((size_t)nrhs * n * 4);
    A->total = o;
}

int check_system(const csk_system& y) {
    if (!y.A || !y.B || !y.Xout || !y.info) return CSK_EINVAL;
    if (y.m < 1 || y.n < 1 || y.d < 1 || y.lda < y.n || y.nrhs < 1 || y.ldb < y.nrhs)
        return CSK_EINVAL;
    if (y.m > INT_MAX || y.n > INT_MAX || y.d > INT_MAX) return CSK_ENOMEM;
    if (y.area && reinterpret_cast<uintptr_t>(y.area) % 256 != 0) return CSK_EINVAL;
    return CSK_OK;
}

// Workspace: sort and Gram-operand scratch (prepare), the descriptor table
// and unit counter (iterate), and the areas of the systems that bring none.
// The sketches and Gram matrices of a batch are formed on up to kPrepLanes
// streams forked from the caller's (each lane with its own sort and Gram
// scratch), so the short launches of small systems overlap.
constexpr int kPrepLanes = 4;

struct BatchLayout {
    size_t sort, gscr, table, counter, total;
    int lanes = 1;                   // prepare lanes the scratch is laid out for
    size_t sort_stride = 0, gscr_stride = 0;
    std::vector<size_t> area;        // offset in ws of each system's area (if it has none)
    std::vector<int> order;          // systems by decreasing d*n
    int64_t mmax, dmax, nmax;
};

int batch_layout(const csk_system* sys, int nsys, bool prepare, bool iterate, BatchLayout* L) {
    L->mmax = L->dmax = L->nmax = 0;
    for (int s = 0; s < nsys; ++s) {
        const int rc = check_system(sys[s]);
        if (rc != CSK_OK) return rc;
        L->mmax = std::max(L->mmax, sys[s].m);
        L->dmax = std::max(L->dmax, sys[s].d);
        L->nmax = std::max(L->nmax, sys[s].n);
    }
    size_t o = 0;
    L->lanes = prepare ? std::min(kPrepLanes, std::max(nsys, 1)) : 1;
    L->sort_stride = prepare ? a256(sort_scratch_bytes(L->mmax, L->dmax)) : 0;
    L->gscr_stride = prepare ? a256(gram_scratch_bytes((int)L->dmax, (int)L->nmax)) : 0;
    L->sort = o;  o += (size_t)L->lanes * L->sort_stride;
    L->gscr = o;  o += (size_t)L->lanes * L->gscr_stride;
    L->table = o; o += iterate ? a256((size_t)nsys * sizeof(BatchSys)) : 0;
    L->counter = o; o += iterate ? 256 : 0;
    L->area.assign(nsys, 0);
    for (int s = 0; s < nsys; ++s) {
        if (sys[s].area) continue;
        AreaLayout A;
        area_layout(sys[s].n, sys[s].d, sys[s].nrhs, &A);
        L->area[s] = o;
        o += A.total;
    }
    L->total = o;
    L->order.resize(nsys);
    std::iota(L->order.begin(), L->order.end(), 0);
    std::stable_sort(L->order.begin(), L->order.end(), [&](int a, int b) {
        return sys[a].d * sys[a].n > sys[b].d * sys[b].n;
    });
    return CSK_OK;
}

char* area_of(const csk_system& y, const BatchLayout& L, int s, char* ws) {
    return y.area ? static_cast<char*>(y.area) : ws + L.area[s];
}

}  // namespace

// ------------------------------------------------------- tuned plans
// Launch shapes (threads per CTA, CTAs) installed by an autotuner for a
// batch signature: the histogram of units (right-hand sides) over
// (floor(log2 d), floor(log2 n)) bins, so batches with the same shape
// distribution share a plan whatever their order.
std::mutex g_plan_mu;
std::map<std::pair<int, uint64_t>, std::pair<int, int>> g_plans;   // (device, signature)

uint64_t batch_signature(const csk_system* sys, int nsys) {
    std::map<std::pair<int, int>, int64_t> hist;
    auto lg = [](int64_t v) { int b = 0; while (v > 1) { v >>= 1; ++b; } return b; };
    for (int s = 0; s < nsys; ++s) hist[{lg(sys[s].d), lg(sys[s].n)}] += sys[s].nrhs;
    uint64_t h = 1469598103934665603ull;               // FNV-1a over the sorted bins
    auto mix = [&h](uint64_t v) {
        for (int i = 0; i < 8; ++i) { h ^= (v >> (8 * i)) & 0xFF; h *= 1099511628211ull; }
    };
    for (const auto& e : hist) {
        mix((uint64_t)e.first.first);
        mix((uint64_t)e.first.second);
        mix((uint64_t)e.second);
    }
    return h;
}

bool lookup_plan(const csk_system* sys, int nsys, int* threads, int* grid) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find({dev, batch_signature(sys, nsys)});
    if (it == g_plans.end()) return false;
    *threads = it->second.first;
    *grid = it->second.second;
    return true;
}

int set_batched_plan(const csk_system* sys, int nsys, int threads, int grid) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CSK_ECUDA;
    const uint64_t key = batch_signature(sys, nsys);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    if (threads == 0 && grid == 0) g_plans.erase({dev, key});
    else g_plans[{dev, key}] = {threads, grid};
    return CSK_OK;
}

uint64_t batched_signature(const csk_system* sys, int nsys) { return batch_signature(sys, nsys); }

size_t batched_workspace_bytes(const csk_system* sys, int nsys, bool prepare, bool iterate) {
    BatchLayout L;
    if (!sys || nsys < 1 || batch_layout(sys, nsys, prepare, iterate, &L) != CSK_OK) return 0;
    return L.total == 0 ? 256 : L.total;
}

size_t batched_area_bytes(int64_t n, int64_t d, int32_t nrhs) {
    AreaLayout A;
    area_layout(n, d, nrhs, &A);
    return A.total;
}

int plan_batched(int64_t dmax, int64_t nmax, int threads_req, int grid_req, int* threads,
                 int* grid, size_t* smem, int* head) {
    DevInfo di;
    if (dev_info(&di) != 0) return CSK_ECUDA;
    size_t need = (size_t)(2 * ((dmax + 3) & ~3) + 2 * ((nmax + 3) & ~3)) * 4;
    if (need + sizeof(BatchShared) + 1024 > (size_t)di.smem_optin) return CSK_EUNSUPPORTED;
    // 256 threads: measured faster than 512 on the 256 x 64 workload (shared
    // memory caps both at the same CTAs per SM)
    int t = threads_req > 0 ? threads_req : 256;
    if (t < 64 || t > 512 || (t & 31)) return CSK_EINVAL;
    // staging of the G rows' heads: what shared memory leaves beside two CTAs
    // per SM (1 KB of each CTA's share is the system's), whole rows when they
    // fit, else a multiple of 4 t values (whole groups of four rows per
    // thread, so every thread keeps its rows whatever H is)
    int64_t H = 0;
    const int64_t share = (int64_t)di.smem_per_sm / 2 - 1024 - (int64_t)sizeof(BatchShared) -
                          (int64_t)need;
    if (share >= 4 * ((dmax + 3) & ~3)) H = (dmax + 3) & ~3;
    else if (share > 0) H = share / 4 / (4 * t) * (4 * t);
    const int64_t cap = ((int64_t)di.smem_optin - 1024 - (int64_t)sizeof(BatchShared) - (int64_t)need) / 4;
    if (H > cap) H = cap / (4 * t) * (4 * t);
    if (H < 0) H = 0;
    need += (size_t)H * 4;
    if (ensure_smem_attr((const void*)k_iterate_batched, need) != cudaSuccess) return CSK_ECUDA;
    int per_sm = 0;
    if (cached_occupancy((const void*)k_iterate_batched, t, need, &per_sm) != cudaSuccess ||
        per_sm < 1)
        return CSK_EUNSUPPORTED;
    *threads = t;
    *grid = grid_req > 0 ? grid_req : per_sm * di.sms;
    *smem = need;
    *head = (int)H;
    return CSK_OK;
}

// Streams and events of the prepare lanes, one set per call in flight
// (kept for reuse): a lane waits for `fork` recorded on the caller's stream,
// and the caller's stream waits for every lane's `join`.
struct PrepLanes {
    int dev = -1;
    cudaStream_t s[kPrepLanes] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kPrepLanes] = {};
};
std::mutex g_lanes_mu;
std::vector<PrepLanes> g_lanes_idle;

void destroy_lanes(PrepLanes& p) {
    for (int l = 0; l < kPrepLanes; ++l) {
        if (p.s[l]) cudaStreamDestroy(p.s[l]);
        if (p.join[l]) cudaEventDestroy(p.join[l]);
    }
    if (p.fork) cudaEventDestroy(p.fork);
}

// A lane set for this device; false when none is idle and the caller's
// stream is being captured into a CUDA graph (no stream is created then: the
// batch is prepared on the caller's stream alone).
bool acquire_lanes(cudaStream_t st, PrepLanes* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    {
        std::lock_guard<std::mutex> lk(g_lanes_mu);
        for (size_t i = 0; i < g_lanes_idle.size(); ++i)
            if (g_lanes_idle[i].dev == dev) {
                *out = g_lanes_idle[i];
                g_lanes_idle.erase(g_lanes_idle.begin() + (std::ptrdiff_t)i);
                return true;
            }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return false;
    PrepLanes p;
    p.dev = dev;
    bool ok = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l < kPrepLanes && ok; ++l)
        ok = cudaStreamCreateWithFlags(&p.s[l], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p.join[l], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        destroy_lanes(p);
        return false;
    }
    *out = p;
    return true;
}

void release_lanes(const PrepLanes& p) {
    std::lock_guard<std::mutex> lk(g_lanes_mu);
    g_lanes_idle.push_back(p);
}

// Sketch and Gram matrix of every system into its area, unit states reset.
// Systems go, largest first, to the lane with the least estimated work so
// far (d^2 n for the Gram matrix plus m n for the sketch); a system's result
// does not depend on its lane.
int prepare_batched(const csk_system* sys, int nsys, const BatchLayout& L, char* w,
                    cudaStream_t st) {
    PrepLanes pl;
    const bool forked = L.lanes > 1 && acquire_lanes(st, &pl);
    const int nl = forked ? L.lanes : 1;
    SortScratch sc[kPrepLanes];
    for (int l = 0; l < nl; ++l)
        carve_sort_scratch(w + L.sort + (size_t)l * L.sort_stride, L.mmax, L.dmax, &sc[l]);
    int rc = CSK_OK;
    if (forked) {
        if (cudaEventRecord(pl.fork, st) != cudaSuccess) rc = CSK_ECUDA;
        for (int l = 0; l < nl && rc == CSK_OK; ++l)
            if (cudaStreamWaitEvent(pl.s[l], pl.fork, 0) != cudaSuccess) rc = CSK_ECUDA;
    }
    double load[kPrepLanes] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < nsys && rc == CSK_OK; ++q) {
        const int i = L.order[q];
        const csk_system& y = sys[i];
        int lane = 0;
        for (int l = 1; l < nl; ++l)
            if (load[l] < load[lane]) lane = l;
        load[lane] += (double)y.d * (double)y.d * (double)y.n + (double)y.m * (double)y.n;
        cudaStream_t ls = forked ? pl.s[lane] : st;
        AreaLayout A;
        area_layout(y.n, y.d, y.nrhs, &A);
        char* a = area_of(y, L, i, w);
        float* At = reinterpret_cast<float*>(a + A.At);
        float* Bt = reinterpret_cast<float*>(a + A.Bt);
        double* N2 = reinterpret_cast<double*>(a + A.N2);
        float* G = reinterpret_cast<float*>(a + A.G);
        if (launch_sketch(CSK_F32, y.A, y.lda, y.m, (int)y.n, y.B, y.ldb, y.nrhs, sc[lane], (int)y.d,
                          y.seed, At, Bt, N2, ls) != cudaSuccess ||
            launch_gram_split_bf16(At, (int)y.d, (int)y.n, N2, G, gram_ld((int)y.d),
                                   w + L.gscr + (size_t)lane * L.gscr_stride, nullptr,
                                   ls) != cudaSuccess ||
            cudaMemsetAsync(a + A.states, 0, (size_t)y.nrhs * sizeof(UnitState), ls) != cudaSuccess)
            rc = CSK_ECUDA;
    }
    if (forked) {
        // join every lane back, also after an error, so no lane work is left
        // unordered with the caller's stream
        for (int l = 0; l < nl; ++l)
            if (cudaEventRecord(pl.join[l], pl.s[l]) != cudaSuccess ||
                cudaStreamWaitEvent(st, pl.join[l], 0) != cudaSuccess)
                rc = CSK_ECUDA;
        release_lanes(pl);
    }
    return rc;
}

// One persistent launch over every unit of the systems (units already
// finished return at once), each running at most `budget` steps (0: to the
// end).
int iterate_batched(const csk_system* sys, int nsys, const csk_params* p, const BatchLog& log,
                    int64_t budget, const BatchLayout& L, char* w, cudaStream_t st) {
    int threads = 0, grid = 0, head = 0;
    size_t smem = 0;
    int t_req = p->threads, g_req = p->grid;
    if (t_req == 0 && g_req == 0) (void)lookup_plan(sys, nsys, &t_req, &g_req);   // tuned shape
    int rc = plan_batched(L.dmax, L.nmax, t_req, g_req, &threads, &grid, &smem, &head);
    if (rc != CSK_OK) return rc;
    std::vector<BatchSys> table(nsys);
    int units = 0, log_unit = -1;
    for (int q = 0; q < nsys; ++q) {
        const int i = L.order[q];
        const csk_system& y = sys[i];
        AreaLayout A;
        area_layout(y.n, y.d, y.nrhs, &A);
        char* a = area_of(y, L, i, w);
        BatchSys& e = table[q];
        e.At = reinterpret_cast<const float*>(a + A.At);
        e.Bt = reinterpret_cast<const float*>(a + A.Bt);
        e.N2 = reinterpret_cast<const double*>(a + A.N2);
        e.G = reinterpret_cast<const float*>(a + A.G);
        e.states = reinterpret_cast<UnitState*>(a + A.states);
        e.rst = reinterpret_cast<float*>(a + A.rst);
        e.xst = reinterpret_cast<float*>(a + A.xst);
        e.X0 = static_cast<const float*>(y.X0);
        e.Xstar = static_cast<const float*>(y.Xstar);
        e.Xout = static_cast<float*>(y.Xout);
        e.info = y.info;
        e.ldg = gram_ld((int)y.d);
        e.d = (int)y.d; e.n = (int)y.n; e.nrhs = y.nrhs; e.unit_begin = units;
        if (i == log.system) log_unit = units + log.rhs;
        units += y.nrhs;
    }
    BatchSys* dtable = reinterpret_cast<BatchSys*>(w + L.table);
    for (int first = 0; first < nsys; first += kTableChunk) {
        TableChunk c;
        c.first = first;
        c.count = std::min(kTableChunk, nsys - first);
        for (int i = 0; i < c.count; ++i) c.e[i] = table[first + i];
        k_write_table<<<1, kTableChunk, 0, st>>>(c, dtable);
        note_launches(1);
    }
    int* counter = reinterpret_cast<int*>(w + L.counter);
    if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return CSK_ECUDA;
    const UnitLog lg = {log.ik, log.ik_len, log.x, log.x_len};
    k_iterate_batched<<<grid, threads, smem, st>>>(dtable, nsys, units, counter, (float)p->tol,
                                                   p->max_iter, p->refresh_every, log_unit, lg,
                                                   budget, head);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? CSK_OK : CSK_ECUDA;
}

int launch_batched(const csk_system* sys, int nsys, const csk_params* p, const BatchLog& log,
                   void* ws, size_t ws_bytes, cudaStream_t st) {
    BatchLayout L;
    int rc = batch_layout(sys, nsys, true, true, &L);
    if (rc != CSK_OK) return rc;
    if (ws_bytes < L.total) return CSK_EINVAL;
    char* w = static_cast<char*>(ws);
    rc = prepare_batched(sys, nsys, L, w, st);
    if (rc != CSK_OK) return rc;
    return iterate_batched(sys, nsys, p, log, 0, L, w, st);
}

int launch_batched_prepare(const csk_system* sys, int nsys, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    BatchLayout L;
    int rc = batch_layout(sys, nsys, true, false, &L);
    if (rc != CSK_OK) return rc;
    for (int s = 0; s < nsys; ++s)
        if (!sys[s].area) return CSK_EINVAL;
    if (ws_bytes < L.total) return CSK_EINVAL;
    return prepare_batched(sys, nsys, L, static_cast<char*>(ws), st);
}

int launch_batched_iterate(const csk_system* sys, int nsys, const csk_params* p,
                           const BatchLog& log, int64_t budget, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    BatchLayout L;
    int rc = batch_layout(sys, nsys, false, true, &L);
    if (rc != CSK_OK) return rc;
    for (int s = 0; s < nsys; ++s)
        if (!sys[s].area) return CSK_EINVAL;
    if (ws_bytes < L.total) return CSK_EINVAL;
    return iterate_batched(sys, nsys, p, log, budget, L, static_cast<char*>(ws), st);
}

}  // namespace csk
