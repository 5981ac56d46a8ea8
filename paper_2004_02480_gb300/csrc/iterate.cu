// iterate.cu -- the maximal-weighted-residual loop of Algorithm 1 on the
// sketch (At, bt), as one persistent cooperative kernel per solve, plus the
// FP64 final check.
//
// Each CTA owns a contiguous block of rows of At.  A step is
//   Phase A  every CTA scores its rows, key_j = r_j^2 / ||At_j||^2, keeps its
//            best (key, row, alpha = r_j / ||At_j||^2) and a partial of the
//            stopping statistic, and publishes them in its slot (release);
//   Phase B  every CTA waits for all slots of this round (acquire, bounded
//            poll count), reduces them in the same fixed order -- so all CTAs
//            take the same decision bit for bit -- tests the stopping rule of
//            Section 3 and applies the projection of Algorithm 1.
// One inter-CTA exchange per step; slots alternate between two banks so a
// fast CTA can never overwrite a slot a slow CTA has still to read.
//
// GEMV path: r = bt - At x is recomputed every step (Algorithm 1 as printed);
// x is replicated in every CTA's shared memory and, when it fits, the CTA's
// rows of At stay resident in shared memory for the whole solve.
// GRAM path: r lives in shared memory, r -= alpha * G[i_k, :] with
// G = At At^T, r_{i_k} = 0 exactly; x is split by columns across CTAs; every
// refresh_every steps r is recomputed as bt - At x with FP64 accumulation.
#include <climits>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace csk {

namespace {

constexpr int kIterThreads = 256;
constexpr int kMaxGrid = 1024;
constexpr int64_t kDefaultSpin = 1ll << 21;

struct RedShared {
    double key[32];
    double alpha[32];
    int32_t idx[32];
    double sum[32];
    double bkey, balpha, bsum;
    int32_t bidx;
};

__device__ __forceinline__ void block_argmax(double& key, double& alpha, int32_t& idx,
                                             RedShared& sr) {
    warp_argmax(key, alpha, idx);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    if (lane == 0) { sr.key[warp] = key; sr.alpha[warp] = alpha; sr.idx[warp] = idx; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        double k = lane < nw ? sr.key[lane] : -1.0;
        double a = lane < nw ? sr.alpha[lane] : 0.0;
        int32_t i = lane < nw ? sr.idx[lane] : INT_MAX;
        warp_argmax(k, a, i);
        if (lane == 0) { sr.bkey = k; sr.balpha = a; sr.bidx = i; }
    }
    __syncthreads();
    key = sr.bkey; alpha = sr.balpha; idx = sr.bidx;
    __syncthreads();
}

__device__ __forceinline__ double block_sum(double v, RedShared& sr) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = lane_id();
    if (lane == 0) sr.sum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        double s = lane < nw ? sr.sum[lane] : 0.0;
        s = warp_sum(s);
        if (lane == 0) sr.bsum = s;
    }
    __syncthreads();
    v = sr.bsum;
    __syncthreads();
    return v;
}

// Publish this CTA's candidate for `round` and gather every CTA's.  Returns
// false when a wait ran out of polls (status CSK_ETIMEOUT recorded).
__device__ bool exchange(Slot* slots, uint32_t round, double& key, double& alpha, int32_t& idx,
                         double& stat, int64_t spin_limit, int fault_inject, csk_info* info,
                         RedShared& sr) {
    const int G = gridDim.x, b = blockIdx.x;
    Slot* bank = slots + (size_t)(round & 1u) * G;
    if (threadIdx.x == 0 && !(fault_inject && b == 0)) {
        bank[b].key = key;
        bank[b].alpha = alpha;
        bank[b].stat = stat;
        bank[b].idx = idx;
        __threadfence();
        st_release_u32(&bank[b].stamp, round + 1u);
    }
    double gk = -1.0, ga = 0.0, gs = 0.0;
    int32_t gi = INT_MAX;
    int timed_out = 0;
    for (int t = threadIdx.x; t < G; t += blockDim.x) {
        int64_t spins = 0;
        while (ld_acquire_u32(&bank[t].stamp) != round + 1u) {
            if (++spins > spin_limit) { timed_out = 1; break; }
        }
        if (timed_out) break;
        // payload read through L2: the line may be stale in L1 from two rounds ago
        const double k2 = __ldcg(&bank[t].key);
        const double a2 = __ldcg(&bank[t].alpha);
        const int32_t i2 = __ldcg(&bank[t].idx);
        gs += __ldcg(&bank[t].stat);
        if (cand_better(k2, i2, gk, gi)) { gk = k2; ga = a2; gi = i2; }
    }
    if (__syncthreads_or(timed_out)) {
        if (threadIdx.x == 0) set_status_once(info, CSK_ETIMEOUT);
        return false;
    }
    block_argmax(gk, ga, gi, sr);
    gs = block_sum(gs, sr);
    key = gk; alpha = ga; idx = gi; stat = gs;
    return true;
}

// Decision shared by every CTA after an exchange (Section 3 stopping rule,
// tested before the step).  Returns a csk_status to stop with, or INT_MIN to
// continue.
__device__ __forceinline__ int decide(double stat, double stop_norm, double tol, int64_t k,
                                      int64_t max_iter, double key) {
    if (stat / stop_norm <= tol) return CSK_OK;
    if (k >= max_iter) return CSK_MAXITER;
    if (key != key || key < 0.0) return CSK_ENUMERIC;   // NaN, or no non-zero row
    if (key == 0.0) return CSK_OK;                       // every residual is exactly 0
    return INT_MIN;
}

__device__ __forceinline__ void finish(csk_info* info, int status, int64_t k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        info->iters = k;
        if (status != CSK_OK) set_status_once(info, status);
    }
}

// ------------------------------------------------------------ GEMV path
template <typename T>
__global__ void __launch_bounds__(kIterThreads, 1)
k_iterate_gemv(IterProblem p, int R, int cache_rows) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ RedShared sr;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = lane_id(), warp = tid >> 5, nw = blockDim.x >> 5;
    const int n = p.n, d = p.d;
    const int r0 = min(d, b * R), r1 = min(d, r0 + R), nr = r1 - r0;
    const int c0 = (int)((int64_t)n * b / G), c1 = (int)((int64_t)n * (b + 1) / G);
    const int npad = (n + 3) & ~3, Rpad = (R + 3) & ~3;
    T* xs = reinterpret_cast<T*>(dsm);
    T* w2s = xs + npad;
    T* bts = w2s + Rpad;
    T* As = bts + Rpad;
    const T* At = static_cast<const T*>(p.At);
    const T* bt = static_cast<const T*>(p.bt);
    const T* x0 = static_cast<const T*>(p.x0);
    const T* xstar = static_cast<const T*>(p.xstar);

    for (int c = tid; c < n; c += blockDim.x) xs[c] = x0 ? x0[c] : T(0);
    for (int q = tid; q < nr; q += blockDim.x) {
        // weight 1/||At_j||^2; -1 marks a zero row (excluded from the argmax),
        // NaN (a NaN/Inf row) is kept so that the failure reaches the decision
        const double N = p.N2[r0 + q];
        w2s[q] = N > 0.0 ? (T)(1.0 / N) : (N == 0.0 ? T(-1) : (T)NAN);
        bts[q] = bt[r0 + q];
    }
    if (cache_rows) {
        for (int64_t e = tid; e < (int64_t)nr * n; e += blockDim.x) {
            const int q = (int)(e / n), c = (int)(e - (int64_t)q * n);
            As[e] = At[(int64_t)(r0 + q) * p.ld + c];
        }
    }
    __syncthreads();
    const double stop_norm = *p.stop_norm;
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    uint32_t round = 0;
    int64_t k = 0;
    int status = CSK_OK;
    for (;;) {
        // Phase A: residuals of the owned rows and the CTA's best row
        double bkey = -1.0, balpha = 0.0, stat = 0.0;
        int32_t bidx = INT_MAX;
        for (int q = warp; q < nr; q += nw) {
            const T* a = cache_rows ? As + (int64_t)q * n : At + (int64_t)(r0 + q) * p.ld;
            T acc = T(0);
            for (int c = lane; c < n; c += 32) acc = fma(a[c], xs[c], acc);
            acc = warp_sum(acc);
            const T r = bts[q] - acc;
            if (lane == 0) {
                const T w = w2s[q];
                if (!(w < T(0))) {
                    const double key = (double)(r * r * w);
                    if (cand_better(key, r0 + q, bkey, bidx)) {
                        bkey = key;
                        balpha = (double)r / p.N2[r0 + q];
                        bidx = r0 + q;
                    }
                }
                if (!xstar) stat += (double)r * (double)r;
            }
        }
        if (xstar)
            for (int c = c0 + tid; c < c1; c += blockDim.x) {
                const double t = (double)xs[c] - (double)xstar[c];
                stat += t * t;
            }
        block_argmax(bkey, balpha, bidx, sr);
        stat = block_sum(stat, sr);
        // Phase B
        if (!exchange(p.slots, round, bkey, balpha, bidx, stat, spin, p.fault_inject, p.info, sr)) {
            status = CSK_ETIMEOUT;
            break;
        }
        ++round;
        const int dec = decide(stat, stop_norm, p.tol, k, p.max_iter, bkey);
        if (dec != INT_MIN) { status = dec; break; }
        if (b == 0 && tid == 0 && p.ik_log && k < p.ik_log_len) p.ik_log[k] = bidx;
        if (b == 0 && p.x_log && k < p.x_log_len)
            for (int c = tid; c < n; c += blockDim.x) static_cast<T*>(p.x_log)[k * n + c] = xs[c];
        // projection onto row i_k: x += alpha * At_{i_k}^T (same in every CTA)
        const T al = (T)balpha;
        const T* arow = At + (int64_t)bidx * p.ld;
        for (int c = tid; c < n; c += blockDim.x) xs[c] = fma(al, arow[c], xs[c]);
        __syncthreads();
        ++k;
    }
    if (b == 0) {
        T* xo = static_cast<T*>(p.x_out);
        for (int c = tid; c < n; c += blockDim.x) xo[c] = xs[c];
    }
    finish(p.info, status, k);
}

// ------------------------------------------------------------ GRAM path
__global__ void __launch_bounds__(kIterThreads, 1)
k_iterate_gram(IterProblem p, int R) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ RedShared sr;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
    const int lane = lane_id(), warp = tid >> 5, nw = blockDim.x >> 5;
    const int n = p.n, d = p.d;
    const int r0 = min(d, b * R), r1 = min(d, r0 + R), nr = r1 - r0;
    const int c0 = (int)((int64_t)n * b / G), c1 = (int)((int64_t)n * (b + 1) / G);
    const int npad = (n + 3) & ~3, Rpad = (R + 3) & ~3;
    float* rs = reinterpret_cast<float*>(dsm);           // Rpad
    float* w2s = rs + Rpad;                              // Rpad
    float* xsl = w2s + Rpad;                             // npad (slice used)
    float* xfull = xsl + npad;                           // npad
    const float* At = static_cast<const float*>(p.At);
    const float* bt = static_cast<const float*>(p.bt);
    const float* x0 = static_cast<const float*>(p.x0);
    const float* xstar = static_cast<const float*>(p.xstar);
    float* xg = static_cast<float*>(p.xg);

    for (int c = c0 + tid; c < c1; c += blockDim.x) xsl[c - c0] = x0 ? x0[c] : 0.0f;
    for (int q = tid; q < nr; q += blockDim.x) {
        const double N = p.N2[r0 + q];
        w2s[q] = N > 0.0 ? (float)(1.0 / N) : (N == 0.0 ? -1.0f : NAN);
    }
    __syncthreads();
    const double stop_norm = *p.stop_norm;
    const int64_t spin = p.spin_limit > 0 ? p.spin_limit : kDefaultSpin;
    const int K = p.refresh_every;
    uint32_t round = 0;
    int64_t k = 0;
    int status = CSK_OK;
    for (;;) {
        if (k == 0 || (K > 0 && k % K == 0)) {
            // FP64 refresh r = bt - At x: gather the x slices first
            for (int c = c0 + tid; c < c1; c += blockDim.x) xg[c] = xsl[c - c0];
            double dk = 0.0, da = 0.0, ds = 0.0;
            int32_t di = 0;
            __syncthreads();
            if (!exchange(p.slots, round, dk, da, di, ds, spin, p.fault_inject, p.info, sr)) {
                status = CSK_ETIMEOUT;
                break;
            }
            ++round;
            for (int c = tid; c < n; c += blockDim.x) xfull[c] = __ldcg(xg + c);
            __syncthreads();
            for (int q = warp; q < nr; q += nw) {
                const float* a = At + (int64_t)(r0 + q) * p.ld;
                double acc = 0.0;
                for (int c = lane; c < n; c += 32) acc = fma((double)a[c], (double)xfull[c], acc);
                acc = warp_sum(acc);
                if (lane == 0) rs[q] = (float)((double)bt[r0 + q] - acc);
            }
            __syncthreads();
        }
        // Phase A
        double bkey = -1.0, balpha = 0.0, stat = 0.0;
        int32_t bidx = INT_MAX;
        for (int q = tid; q < nr; q += blockDim.x) {
            const float r = rs[q], w = w2s[q];
            if (!(w < 0.0f)) {
                const double key = (double)(r * r * w);
                if (cand_better(key, r0 + q, bkey, bidx)) {
                    bkey = key;
                    balpha = (double)r / p.N2[r0 + q];
                    bidx = r0 + q;
                }
            }
            if (!xstar) stat += (double)r * (double)r;
        }
        if (xstar)
            for (int c = c0 + tid; c < c1; c += blockDim.x) {
                const double t = (double)xsl[c - c0] - (double)xstar[c];
                stat += t * t;
            }
        block_argmax(bkey, balpha, bidx, sr);
        stat = block_sum(stat, sr);
        if (!exchange(p.slots, round, bkey, balpha, bidx, stat, spin, p.fault_inject, p.info, sr)) {
            status = CSK_ETIMEOUT;
            break;
        }
        ++round;
        const int dec = decide(stat, stop_norm, p.tol, k, p.max_iter, bkey);
        if (dec != INT_MIN) { status = dec; break; }
        if (b == 0 && tid == 0 && p.ik_log && k < p.ik_log_len) p.ik_log[k] = bidx;
        if (p.x_log && k < p.x_log_len)
            for (int c = c0 + tid; c < c1; c += blockDim.x)
                static_cast<float*>(p.x_log)[k * n + c] = xsl[c - c0];
        // r -= alpha G[i_k, :] on the owned rows, r_{i_k} = 0 exactly;
        // x slice += alpha At_{i_k}
        const float al = (float)balpha;
        const float* grow = p.G + (int64_t)bidx * p.ldg;
        for (int q = tid; q < nr; q += blockDim.x) {
            const int j = r0 + q;
            rs[q] = (j == bidx) ? 0.0f : fmaf(-al, grow[j], rs[q]);
        }
        const float* arow = At + (int64_t)bidx * p.ld;
        for (int c = c0 + tid; c < c1; c += blockDim.x) xsl[c - c0] = fmaf(al, arow[c], xsl[c - c0]);
        __syncthreads();
        ++k;
    }
    float* xo = static_cast<float*>(p.x_out);
    for (int c = c0 + tid; c < c1; c += blockDim.x) xo[c] = xsl[c - c0];
    finish(p.info, status, k);
}

// --------------------------------------------------------- final check
constexpr int kFinalThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kFinalThreads)
k_final_rows(const T* __restrict__ At, int64_t ld, int d, int n, const T* __restrict__ bt,
             const double* __restrict__ N2, const T* __restrict__ x, double* __restrict__ part) {
    __shared__ RedShared sr;
    const int lane = lane_id();
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double rr = 0.0, bb = 0.0, empty = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < d; j += nwarps) {
        double s = 0.0;
        for (int c = lane; c < n; c += 32) s = fma((double)At[j * ld + c], (double)x[c], s);
        s = warp_sum(s);
        if (lane == 0) {
            const double r = (double)bt[j] - s;
            rr += r * r;
            bb += (double)bt[j] * (double)bt[j];
            empty += (N2[j] > 0.0) ? 0.0 : 1.0;
        }
    }
    rr = block_sum(rr, sr);
    bb = block_sum(bb, sr);
    empty = block_sum(empty, sr);
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
    __shared__ RedShared sr;
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
    rr = block_sum(rr, sr);
    bb = block_sum(bb, sr);
    empty = block_sum(empty, sr);
    ee = block_sum(ee, sr);
    ss = block_sum(ss, sr);
    if (threadIdx.x == 0) {
        info->resid = sqrt(rr / bb);
        info->rse = xstar ? ee / ss : (double)NAN;
        info->empty_rows = (int32_t)empty;
    }
}

int final_blocks(int d) {
    DevInfo di;
    dev_info(&di);
    int64_t blocks = ((int64_t)d + 7) / 8;
    const int64_t cap = (int64_t)(di.sms > 0 ? di.sms : 1) * 4;
    return (int)(blocks < cap ? blocks : cap);
}

}  // namespace

// ------------------------------------------------------------ host side
int plan_iterate(int path, int dtype, int d, int n, int grid_req, IterConfig* cfg) {
    DevInfo di;
    if (dev_info(&di) != 0) return CSK_ECUDA;
    const int s = dtype == CSK_F64 ? 8 : 4;
    const size_t budget = (size_t)di.smem_optin - 2048;   // static shared + slack
    int G = grid_req > 0 ? grid_req : di.sms;
    if (G > kMaxGrid) G = kMaxGrid;
    if (G > d) G = d;
    if (G < 1) G = 1;
    if (grid_req <= 0) {
        // small problems: fewer CTAs, cheaper exchange
        const int64_t cells = (int64_t)d * n;
        int64_t want = (cells + 16383) / 16384;          // ~16K cells of At per CTA
        if (want < 1) want = 1;
        if (want < G) G = (int)want;
    }
    const int R = (d + G - 1) / G;
    const int npad = (n + 3) & ~3, Rpad = (R + 3) & ~3;
    cfg->grid = G;
    cfg->threads = kIterThreads;
    cfg->rows_per_cta = R;
    if (path == CSK_RESID_GRAM) {
        cfg->cache_rows = 0;
        cfg->smem = (size_t)(2 * Rpad + 2 * npad) * 4;
    } else {
        const size_t base = (size_t)(npad + 2 * Rpad) * s;
        const size_t rows = (size_t)R * n * s;
        cfg->cache_rows = (base + rows <= budget) ? 1 : 0;
        cfg->smem = base + (cfg->cache_rows ? rows : 0);
    }
    if (cfg->smem > budget) return CSK_EUNSUPPORTED;
    return CSK_OK;
}

cudaError_t launch_iterate(int path, const IterProblem& p, const IterConfig& cfg, cudaStream_t st) {
    void* fn;
    if (path == CSK_RESID_GRAM) fn = (void*)k_iterate_gram;
    else if (p.dtype == CSK_F64) fn = (void*)k_iterate_gemv<double>;
    else fn = (void*)k_iterate_gemv<float>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, cfg.threads, cfg.smem);
    if (e != cudaSuccess) return e;
    DevInfo di;
    dev_info(&di);
    if ((int64_t)per_sm * di.sms < cfg.grid) return cudaErrorCooperativeLaunchTooLarge;
    IterProblem pc = p;
    int R = cfg.rows_per_cta, cache = cfg.cache_rows;
    void* args_gemv[] = {&pc, &R, &cache};
    void* args_gram[] = {&pc, &R};
    e = cudaLaunchCooperativeKernel(fn, dim3(cfg.grid), dim3(cfg.threads),
                                    path == CSK_RESID_GRAM ? args_gram : args_gemv, cfg.smem, st);
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
