// api.cu -- the C ABI of libcsk (include/csk.h): argument checks, workspace
// layout and the stream-ordered launch sequence of each entry point.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace csk {

namespace {
std::atomic<int64_t> g_launches{0};
constexpr int kMaxDevices = 64;
DevInfo g_dev[kMaxDevices];
std::once_flag g_dev_once[kMaxDevices];

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

__global__ void k_info_init(csk_info* info, int path, int rows, int grid) {
    info->status = CSK_OK;
    info->path = path;
    info->iters = 0;
    info->rse = (double)NAN;
    info->resid = (double)NAN;
    info->rows = rows;
    info->empty_rows = 0;
    info->grid = grid;
    info->reserved0 = 0;
    info->reserved1 = 0.0;
    info->reserved2 = 0.0;
}

// Workspace of csk_solve, in order (each piece 256-byte aligned):
//   sort scratch | At (d x n) | bt (d) | N2 (rows) | stop norm (8 doubles) |
//   exchange mailboxes (2 x grid x grid) | x gather (n) | final-check partials |
//   G (d x d, GRAM) | Gram operand scratch (GRAM)

struct SolveLayout {
    size_t sort, At, bt, N2, norm, slots, xg, part, fpart, G, gscr, total;
};

void solve_layout(int64_t m, int64_t n, int dtype, int64_t d, int path, SolveLayout* L) {
    const size_t s = dtype == CSK_F64 ? 8 : 4;
    const int64_t rows = d > 0 ? d : m;
    size_t o = 0;
    L->sort = o;  o += d > 0 ? align256(sort_scratch_bytes(m, d)) : 0;
    L->At = o;    o += d > 0 ? align256((size_t)d * n * s) : 0;
    L->bt = o;    o += d > 0 ? align256((size_t)d * s) : 0;
    L->N2 = o;    o += align256((size_t)rows * 8);
    L->norm = o;  o += 256;
    L->slots = o; o += align256(exchange_bytes(kMaxIterGrid));
    L->xg = o;    o += align256((size_t)n * s);
    L->part = o;  o += align256(final_check_partials((int)rows) * 8);
    L->fpart = o; o += align256((size_t)kMaxIterGrid * 8);
    L->G = o;     o += path == CSK_RESID_GRAM ? align256((size_t)rows * gram_ld((int)rows) * 4) : 0;
    L->gscr = o;  o += path == CSK_RESID_GRAM ? align256(gram_scratch_bytes((int)rows, (int)n)) : 0;
    L->total = o;
}

// AUTO: GEMV while the sketch fits on chip across the SMs (shared memory or
// registers, ~24 MB), else GRAM (FP32 only; an unsketched A stays GEMV).
int resolve_path(int path, int dtype, int64_t d, int64_t n) {
    if (path != CSK_RESID_AUTO) return path;
    if (dtype != CSK_F32 || d == 0) return CSK_RESID_GEMV;
    return d * n * 4 <= (int64_t)24 << 20 ? CSK_RESID_GEMV : CSK_RESID_GRAM;
}

int check_solve_args(int64_t m, int64_t n, int64_t lda, int32_t dtype, const csk_params* params,
                     const void* ws) {
    if (m < 1 || n < 1 || lda < n) return CSK_EINVAL;
    if (dtype != CSK_F32 && dtype != CSK_F64) return CSK_EINVAL;
    const int64_t d = params->d;
    if (d < 0 || !(params->tol >= 0.0) || params->max_iter < 0) return CSK_EINVAL;
    if (params->ik_log_len < 0 || (params->ik_log_len > 0 && !params->ik_log)) return CSK_EINVAL;
    if (params->x_log_len < 0 || (params->x_log_len > 0 && !params->x_log)) return CSK_EINVAL;
    if (params->path < CSK_RESID_GEMV || params->path > CSK_RESID_UPDATE) return CSK_EINVAL;
    if (params->grid < 0 || params->refresh_every < 0) return CSK_EINVAL;
    if (params->gemv_variant < 0 || params->gemv_variant > 3) return CSK_EINVAL;
    if (params->fused != 0 && params->fused != 1) return CSK_EINVAL;
    if (params->fused && (params->d == 0 || resolve_path(params->path, dtype, params->d, n) !=
                                                CSK_RESID_GEMV))
        return CSK_EUNSUPPORTED;
    if (m > INT_MAX || n > INT_MAX || d > INT_MAX) return CSK_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    const int path = resolve_path(params->path, dtype, d, n);
    if (path == CSK_RESID_GRAM && dtype != CSK_F32) return CSK_EUNSUPPORTED;
    if (path == CSK_RESID_GRAM && d == 0) return CSK_EUNSUPPORTED;   // an m x m Gram is pointless
    return CSK_OK;
}

// Device staging of csk_solve_host: A (m x n packed), b, x0, x*, x, info.
struct HostStaging {
    size_t A, b, x0, xs, x, info, total;
};
void host_staging(int64_t m, int64_t n, int dtype, HostStaging* H) {
    const size_t s = dtype == CSK_F64 ? 8 : 4;
    size_t o = 0;
    H->A = o;    o += align256((size_t)m * n * s);
    H->b = o;    o += align256((size_t)m * s);
    H->x0 = o;   o += align256((size_t)n * s);
    H->xs = o;   o += align256((size_t)n * s);
    H->x = o;    o += align256((size_t)n * s);
    H->info = o; o += 256;
    H->total = o;
}

// Host-to-device copies of one csk_solve_host problem; A is packed to leading
// dimension n on the device (one linear copy when it already is).
cudaError_t copy_in(const void* A_host, int64_t m, int64_t n, int64_t lda, const void* b_host,
                    const void* x0_host, const void* xs_host, size_t s, void* A, void* b,
                    void* x0, void* xs, cudaStream_t st) {
    cudaError_t e = lda == n
        ? cudaMemcpyAsync(A, A_host, (size_t)m * n * s, cudaMemcpyHostToDevice, st)
        : cudaMemcpy2DAsync(A, (size_t)n * s, A_host, (size_t)lda * s, (size_t)n * s, (size_t)m,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b, b_host, (size_t)m * s, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && x0)
        e = cudaMemcpyAsync(x0, x0_host, (size_t)n * s, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && xs)
        e = cudaMemcpyAsync(xs, xs_host, (size_t)n * s, cudaMemcpyHostToDevice, st);
    return e;
}

inline void record(const csk_params* p, int i, cudaStream_t st) {
    if (p->stage_events[i]) cudaEventRecord(static_cast<cudaEvent_t>(p->stage_events[i]), st);
}

int solve_enqueue(const void* A, int64_t m, int64_t n, int64_t lda, const void* b, int32_t dtype,
                  const csk_params* params, const void* x0, const void* x_star, void* x_out,
                  csk_info* info, void* ws, const SolveLayout& L, cudaStream_t st) {
    const int64_t d = params->d;
    const int path = resolve_path(params->path, dtype, d, n);
    const int rows = (int)(d > 0 ? d : m);
    IterConfig cfg;
    const int64_t ld_it = d > 0 ? n : lda;
    const int vlen = dtype == CSK_F64 ? 2 : 4;   // elements per 16-byte chunk
    const bool vec_ok = (ld_it % vlen == 0) &&
                        (d > 0 || reinterpret_cast<uintptr_t>(A) % 16 == 0);
    int rc = plan_iterate(path, dtype, rows, (int)n, params->grid, params->gemv_variant, vec_ok,
                          &cfg);
    if (rc != CSK_OK) return rc;
    if (cfg.grid > kMaxIterGrid) return CSK_EUNSUPPORTED;

    char* w = static_cast<char*>(ws);
    const void* At;
    const void* bt;
    int64_t ld;
    double* N2 = reinterpret_cast<double*>(w + L.N2);
    int fcap = 0;
    size_t fsmem = 0;
    if (params->fused) {
        rc = plan_fused(dtype, m, (int)d, (int)n, cfg, A, lda, &fcap, &fsmem);
        if (rc != CSK_OK) return rc;
    }
    record(params, 0, st);
    k_info_init<<<1, 1, 0, st>>>(info, path, rows, cfg.grid);
    note_launches(1);
    if (params->fused) {
        // the whole loop, sketch included, in one cooperative kernel
        Slot* slots = reinterpret_cast<Slot*>(w + L.slots);
        if (cudaMemsetAsync(slots, 0, exchange_bytes(cfg.grid), st) != cudaSuccess) return CSK_ECUDA;
        record(params, 1, st);
        record(params, 2, st);
        SortScratch s;
        carve_sort_scratch(w + L.sort, m, d, &s);
        FusedArgs fa;
        fa.A = A; fa.lda = lda; fa.m = m; fa.b = b; fa.seed = params->seed;
        fa.h = reinterpret_cast<uint16_t*>(s.perm_tmp);
        fa.perm = s.perm;
        fa.off = s.off;
        fa.part = reinterpret_cast<double*>(w + L.fpart);
        IterProblem p;
        p.dtype = dtype;
        p.At = w + L.At; p.ld = n; p.d = rows; p.n = (int)n;
        p.bt = w + L.bt; p.N2 = N2;
        p.x0 = x0; p.xstar = x_star; p.x_out = x_out;
        p.stop_norm = nullptr;
        p.slots = slots;
        p.xg = w + L.xg;
        p.G = nullptr; p.ldg = 0;
        p.refresh_every = params->refresh_every;
        p.ik_log = params->ik_log; p.ik_log_len = params->ik_log_len;
        p.x_log = params->x_log; p.x_log_len = params->x_log_len;
        p.tol = params->tol; p.max_iter = params->max_iter;
        p.spin_limit = params->spin_limit; p.fault_inject = params->fault_inject;
        p.info = info;
        if (launch_fused(dtype, p, cfg, fa, fcap, fsmem, st) != cudaSuccess) return CSK_ECUDA;
        record(params, 3, st);
        if (launch_final_check(dtype, w + L.At, n, rows, (int)n, w + L.bt, N2, x_out, x_star,
                               reinterpret_cast<double*>(w + L.part), info, st) != cudaSuccess)
            return CSK_ECUDA;
        record(params, 4, st);
        return CSK_OK;
    }
    if (d > 0) {
        SortScratch s;
        carve_sort_scratch(w + L.sort, m, d, &s);
        if (launch_sketch(dtype, A, lda, m, (int)n, b, 1, 1, s, (int)d, params->seed, w + L.At,
                          w + L.bt, N2, st) != cudaSuccess)
            return CSK_ECUDA;
        At = w + L.At;
        bt = w + L.bt;
        ld = n;
    } else {
        if (launch_row_norms(dtype, A, lda, (int)m, (int)n, N2, st) != cudaSuccess) return CSK_ECUDA;
        At = A;
        bt = b;
        ld = lda;
    }
    record(params, 1, st);
    double* stop_norm = reinterpret_cast<double*>(w + L.norm);
    if (launch_norm2(dtype, x_star ? x_star : bt, x_star ? n : rows, stop_norm, st) != cudaSuccess)
        return CSK_ECUDA;
    Slot* slots = reinterpret_cast<Slot*>(w + L.slots);
    if (cudaMemsetAsync(slots, 0, exchange_bytes(cfg.grid), st) != cudaSuccess)
        return CSK_ECUDA;
    float* G = nullptr;
    if (path == CSK_RESID_GRAM) {
        G = reinterpret_cast<float*>(w + L.G);
        if (launch_gram_split_bf16(static_cast<const float*>(At), rows, (int)n, N2, G, gram_ld(rows),
                                   w + L.gscr, info, st) != cudaSuccess)
            return CSK_ECUDA;
    }
    record(params, 2, st);
    IterProblem p;
    p.dtype = dtype;
    p.At = At; p.ld = ld; p.d = rows; p.n = (int)n;
    p.bt = bt; p.N2 = N2;
    p.x0 = x0; p.xstar = x_star; p.x_out = x_out;
    p.stop_norm = stop_norm;
    p.slots = slots;
    p.xg = w + L.xg;
    p.G = G; p.ldg = gram_ld(rows);
    p.refresh_every = params->refresh_every;
    p.ik_log = params->ik_log; p.ik_log_len = params->ik_log_len;
    p.x_log = params->x_log; p.x_log_len = params->x_log_len;
    p.tol = params->tol; p.max_iter = params->max_iter;
    p.spin_limit = params->spin_limit; p.fault_inject = params->fault_inject;
    p.info = info;
    if (launch_iterate(path, p, cfg, st) != cudaSuccess) return CSK_ECUDA;
    record(params, 3, st);
    if (launch_final_check(dtype, At, ld, rows, (int)n, bt, N2, x_out, x_star,
                           reinterpret_cast<double*>(w + L.part), info, st) != cudaSuccess)
        return CSK_ECUDA;
    record(params, 4, st);
    return CSK_OK;
}
// Copy stream and events of csk_solve_host_many, created once per device and
// reused: an idle set is taken at the start of a call and returned at its end
// (calls running at the same time on one device each get a set of their own).
struct CopyRes {
    int dev = -1;
    cudaStream_t cp = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    cudaEvent_t freed[2] = {nullptr, nullptr};
};
std::mutex g_res_mu;
std::vector<CopyRes> g_res_idle;

void destroy_copy_res(CopyRes& r) {
    for (int i = 0; i < 2; ++i) {
        if (r.copied[i]) cudaEventDestroy(r.copied[i]);
        if (r.freed[i]) cudaEventDestroy(r.freed[i]);
    }
    if (r.cp) cudaStreamDestroy(r.cp);
}

cudaError_t acquire_copy_res(CopyRes* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        for (size_t i = 0; i < g_res_idle.size(); ++i)
            if (g_res_idle[i].dev == dev) {
                *out = g_res_idle[i];
                g_res_idle.erase(g_res_idle.begin() + (std::ptrdiff_t)i);
                return cudaSuccess;
            }
    }
    CopyRes r;
    r.dev = dev;
    e = cudaStreamCreateWithFlags(&r.cp, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&r.copied[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.freed[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        destroy_copy_res(r);
        return e;
    }
    *out = r;
    return cudaSuccess;
}

void release_copy_res(const CopyRes& r) {
    std::lock_guard<std::mutex> lk(g_res_mu);
    g_res_idle.push_back(r);
}
}  // namespace

void note_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int check_stream_device(cudaStream_t st) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return CSK_ECUDA;
    if (st == nullptr) return CSK_OK;
    // A stream being captured into a CUDA graph cannot be queried for its
    // device (the query would invalidate the capture); skip the check then.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return CSK_EINVAL;
    if (cap != cudaStreamCaptureStatusNone) return CSK_OK;
    int sd = -1;
    if (cudaStreamGetDevice(st, &sd) != cudaSuccess) return CSK_EINVAL;
    return sd == cur ? CSK_OK : CSK_EINVAL;
}


namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_set;                  // largest set so far
std::map<std::tuple<int, const void*, int, size_t>, int> g_occupancy;
}  // namespace

cudaError_t ensure_smem_attr(const void* fn, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto key = std::make_pair(dev, fn);
    auto it = g_smem_set.find(key);
    if (it != g_smem_set.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) g_smem_set[key] = smem;
    return e;
}

cudaError_t cached_occupancy(const void* fn, int threads, size_t smem, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto key = std::make_tuple(dev, fn, threads, smem);
    auto it = g_occupancy.find(key);
    if (it != g_occupancy.end()) { *per_sm = it->second; return cudaSuccess; }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
    if (e == cudaSuccess) g_occupancy[key] = *per_sm;
    return e;
}

int dev_info(DevInfo* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    std::call_once(g_dev_once[dev], [dev] {
        DevInfo d;
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&d.coop, cudaDevAttrCooperativeLaunch, dev);
        g_dev[dev] = d;
    });
    *out = g_dev[dev];
    return out->sms > 0 ? 0 : -1;
}

}  // namespace csk

using namespace csk;

extern "C" {

void csk_params_default(csk_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tol = 1e-6;
    p->max_iter = 20000;
    p->path = CSK_RESID_GEMV;
}

const char* csk_strerror(int status) {
    switch (status) {
        case CSK_OK: return "CSK_OK";
        case CSK_MAXITER: return "CSK_MAXITER: step cap reached";
        case CSK_INPROGRESS: return "CSK_INPROGRESS: step budget of this call ran out";
        case CSK_EINVAL: return "CSK_EINVAL: invalid argument";
        case CSK_ENOMEM: return "CSK_ENOMEM: size out of supported range";
        case CSK_ETIMEOUT: return "CSK_ETIMEOUT: inter-CTA wait exceeded its poll limit";
        case CSK_ENUMERIC: return "CSK_ENUMERIC: NaN/Inf residual or no non-zero row";
        case CSK_ECUDA: return "CSK_ECUDA: CUDA runtime error";
        case CSK_EUNSUPPORTED: return "CSK_EUNSUPPORTED: not supported by this library";
        default: return "unknown csk status";
    }
}

int csk_version(void) { return 200; }

int64_t csk_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

size_t csk_sketch_workspace_size(int64_t m, int64_t d) {
    if (m < 1 || d < 1) return 0;
    return sort_scratch_bytes(m, d);
}

int csk_sketch(const void* A, int64_t m, int64_t n, int64_t lda, const void* B, int64_t ldb,
               int32_t nrhs, int32_t dtype, int64_t d, uint64_t seed, void* At, void* Bt,
               double* norms2_out, int32_t* perm_out, int32_t* off_out, void* ws,
               size_t ws_bytes, void* stream) {
    if (!A || !At || !ws) return CSK_EINVAL;
    if (m < 1 || n < 1 || d < 1 || lda < n || nrhs < 0) return CSK_EINVAL;
    if (dtype != CSK_F32 && dtype != CSK_F64) return CSK_EINVAL;
    if (nrhs > 0 && (!B || !Bt || ldb < nrhs)) return CSK_EINVAL;
    if (m > INT_MAX || n > INT_MAX || d > INT_MAX) return CSK_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    if (ws_bytes < csk_sketch_workspace_size(m, d)) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    SortScratch s;
    carve_sort_scratch(ws, m, d, &s);
    if (perm_out) s.perm = perm_out;
    if (off_out) s.off = off_out;
    if (launch_sketch(dtype, A, lda, m, (int)n, nrhs > 0 ? B : nullptr, ldb, nrhs, s, (int)d, seed,
                      At, Bt, norms2_out, st) != cudaSuccess)
        return CSK_ECUDA;
    return CSK_OK;
}

size_t csk_gram_workspace_size(int64_t d, int64_t n) {
    if (d < 1 || n < 1 || d > INT_MAX || n > INT_MAX) return 0;
    return align256(gram_scratch_bytes((int)d, (int)n));
}

int csk_gram(const float* At, int64_t d, int64_t n, const double* norms2, float* G, int64_t ldg,
             csk_info* info, void* ws, size_t ws_bytes, void* stream) {
    if (!At || !G || !ws) return CSK_EINVAL;
    if (d < 1 || n < 1 || ldg < d) return CSK_EINVAL;
    if (d > INT_MAX || n > INT_MAX) return CSK_ENOMEM;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    if (ws_bytes < csk_gram_workspace_size(d, n)) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    if (launch_gram_split_bf16(At, (int)d, (int)n, norms2, G, ldg, ws, info, st) != cudaSuccess)
        return CSK_ECUDA;
    return CSK_OK;
}

size_t csk_solve_batched_workspace_size(const csk_system* sys, int32_t nsys) {
    return batched_workspace_bytes(sys, nsys, true, true);
}

int csk_solve_batched(const csk_system* sys, int32_t nsys, const csk_params* params, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!sys || nsys < 1 || !params || !ws) return CSK_EINVAL;
    if (!(params->tol >= 0.0) || params->max_iter < 0 || params->refresh_every < 0 ||
        params->grid < 0 || params->threads < 0)
        return CSK_EINVAL;
    if (params->ik_log_len < 0 || (params->ik_log_len > 0 && !params->ik_log)) return CSK_EINVAL;
    if (params->x_log_len < 0 || (params->x_log_len > 0 && !params->x_log)) return CSK_EINVAL;
    BatchLog log;
    if (params->ik_log_len > 0 || params->x_log_len > 0) {
        if (params->log_system < 0 || params->log_system >= nsys || params->log_rhs < 0 ||
            params->log_rhs >= sys[params->log_system].nrhs)
            return CSK_EINVAL;
        log.system = params->log_system;
        log.rhs = params->log_rhs;
        log.ik = params->ik_log_len > 0 ? params->ik_log : nullptr;
        log.ik_len = params->ik_log_len;
        log.x = params->x_log_len > 0 ? static_cast<float*>(params->x_log) : nullptr;
        log.x_len = params->x_log_len;
    }
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    return launch_batched(sys, nsys, params, log, ws, ws_bytes, st);
}

size_t csk_batched_area_size(int64_t n, int64_t d, int32_t nrhs) {
    if (n < 1 || d < 1 || nrhs < 1 || n > INT_MAX || d > INT_MAX) return 0;
    return batched_area_bytes(n, d, nrhs);
}

size_t csk_batched_prepare_workspace_size(const csk_system* sys, int32_t nsys) {
    return batched_workspace_bytes(sys, nsys, true, false);
}

size_t csk_batched_iterate_workspace_size(const csk_system* sys, int32_t nsys) {
    return batched_workspace_bytes(sys, nsys, false, true);
}

int csk_batched_prepare(const csk_system* sys, int32_t nsys, void* ws, size_t ws_bytes,
                        void* stream) {
    if (!sys || nsys < 1 || !ws) return CSK_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    return launch_batched_prepare(sys, nsys, ws, ws_bytes, st);
}

int csk_batched_iterate(const csk_system* sys, int32_t nsys, const csk_params* params,
                        int64_t step_budget, void* ws, size_t ws_bytes, void* stream) {
    if (!sys || nsys < 1 || !params || !ws || step_budget < 0) return CSK_EINVAL;
    if (!(params->tol >= 0.0) || params->max_iter < 0 || params->refresh_every < 0 ||
        params->grid < 0 || params->threads < 0)
        return CSK_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    BatchLog log;
    if (params->ik_log_len > 0 || params->x_log_len > 0) {
        if (params->log_system < 0 || params->log_system >= nsys || params->log_rhs < 0 ||
            params->log_rhs >= sys[params->log_system].nrhs ||
            (params->ik_log_len > 0 && !params->ik_log) || (params->x_log_len > 0 && !params->x_log))
            return CSK_EINVAL;
        log.system = params->log_system;
        log.rhs = params->log_rhs;
        log.ik = params->ik_log_len > 0 ? params->ik_log : nullptr;
        log.ik_len = params->ik_log_len;
        log.x = params->x_log_len > 0 ? static_cast<float*>(params->x_log) : nullptr;
        log.x_len = params->x_log_len;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    return launch_batched_iterate(sys, nsys, params, log, step_budget, ws, ws_bytes, st);
}

int csk_solve_batched_set_plan(const csk_system* sys, int32_t nsys, int32_t threads,
                               int32_t grid) {
    if (!sys || nsys < 1 || threads < 0 || grid < 0) return CSK_EINVAL;
    if ((threads == 0) != (grid == 0)) return CSK_EINVAL;
    if (threads != 0 && (threads < 64 || threads > 512 || (threads & 31))) return CSK_EINVAL;
    for (int32_t s = 0; s < nsys; ++s)
        if (sys[s].d < 1 || sys[s].n < 1 || sys[s].nrhs < 1) return CSK_EINVAL;
    return set_batched_plan(sys, nsys, threads, grid);
}

uint64_t csk_solve_batched_signature(const csk_system* sys, int32_t nsys) {
    if (!sys || nsys < 1) return 0;
    return batched_signature(sys, nsys);
}

int csk_info_sync(const csk_info* info_dev, csk_info* info_host, void* stream) {
    if (!info_dev || !info_host) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(info_host, info_dev, sizeof(csk_info), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CSK_ECUDA;
    return info_host->status;
}

size_t csk_workspace_size(int64_t m, int64_t n, int64_t d, int32_t nrhs, int32_t dtype,
                          int32_t resid) {
    if (m < 1 || n < 1 || d < 0 || nrhs < 0) return 0;
    if (dtype != CSK_F32 && dtype != CSK_F64) return 0;
    if (resid < CSK_RESID_GEMV || resid > CSK_RESID_UPDATE) return 0;
    csk_params p;
    csk_params_default(&p);
    p.d = d;
    p.path = resid;
    size_t need = csk_solve_workspace_size(m, n, dtype, &p);
    if (d >= 1) need = std::max(need, csk_sketch_workspace_size(m, d));
    if (dtype == CSK_F32 && d >= 1 && nrhs >= 1) {
        csk_system y;
        std::memset(&y, 0, sizeof(y));
        const uintptr_t any = 256;          // the size depends on shapes only
        y.A = y.B = reinterpret_cast<const void*>(any);
        y.Xout = reinterpret_cast<void*>(any);
        y.info = reinterpret_cast<csk_info*>(any);
        y.m = m; y.n = n; y.lda = n; y.ldb = nrhs; y.nrhs = nrhs; y.d = d;
        need = std::max(need, batched_workspace_bytes(&y, 1, true, true));
    }
    return need;
}

size_t csk_exchange_floor_workspace_size(int32_t grid) {
    if (grid < 1 || grid > kMaxIterGrid) return 0;
    return align256(exchange_bytes(grid)) + 256;
}

int csk_exchange_floor(int32_t grid, int64_t rounds, void* ws, size_t ws_bytes, void* stream) {
    if (grid < 1 || grid > kMaxIterGrid || rounds < 1 || !ws) return CSK_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CSK_EINVAL;
    if (ws_bytes < csk_exchange_floor_workspace_size(grid)) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    char* w = static_cast<char*>(ws);
    Slot* slots = reinterpret_cast<Slot*>(w);
    csk_info* info = reinterpret_cast<csk_info*>(w + align256(exchange_bytes(grid)));
    if (cudaMemsetAsync(w, 0, align256(exchange_bytes(grid)) + sizeof(csk_info), st) != cudaSuccess)
        return CSK_ECUDA;
    return launch_exchange_probe(grid, rounds, slots, info, st) == cudaSuccess ? CSK_OK : CSK_ECUDA;
}

size_t csk_solve_workspace_size(int64_t m, int64_t n, int32_t dtype, const csk_params* params) {
    if (!params || m < 1 || n < 1 || params->d < 0) return 0;
    if (dtype != CSK_F32 && dtype != CSK_F64) return 0;
    SolveLayout L;
    solve_layout(m, n, dtype, params->d, resolve_path(params->path, dtype, params->d, n), &L);
    return L.total;
}

int csk_solve(const void* A, int64_t m, int64_t n, int64_t lda, const void* b, int32_t dtype,
              const csk_params* params, const void* x0, const void* x_star, void* x_out,
              csk_info* info, void* ws, size_t ws_bytes, void* stream) {
    if (!A || !b || !params || !x_out || !info || !ws) return CSK_EINVAL;
    int rc = check_solve_args(m, n, lda, dtype, params, ws);
    if (rc != CSK_OK) return rc;
    SolveLayout L;
    solve_layout(m, n, dtype, params->d, resolve_path(params->path, dtype, params->d, n), &L);
    if (ws_bytes < L.total) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    return solve_enqueue(A, m, n, lda, b, dtype, params, x0, x_star, x_out, info, ws, L, st);
}

size_t csk_solve_host_workspace_size(int64_t m, int64_t n, int32_t dtype, const csk_params* params) {
    const size_t inner = csk_solve_workspace_size(m, n, dtype, params);
    if (inner == 0) return 0;
    HostStaging H;
    host_staging(m, n, dtype, &H);
    return H.total + inner;
}

int csk_solve_host(const void* A_host, int64_t m, int64_t n, int64_t lda, const void* b_host,
                   int32_t dtype, const csk_params* params, const void* x0_host,
                   const void* x_star_host, void* x_out_host, csk_info* info_host, void* ws,
                   size_t ws_bytes, void* stream) {
    if (!A_host || !b_host || !params || !x_out_host || !info_host || !ws) return CSK_EINVAL;
    int rc = check_solve_args(m, n, lda, dtype, params, ws);
    if (rc != CSK_OK) return rc;
    HostStaging H;
    host_staging(m, n, dtype, &H);
    SolveLayout L;
    solve_layout(m, n, dtype, params->d, resolve_path(params->path, dtype, params->d, n), &L);
    if (ws_bytes < H.total + L.total) return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    const size_t s = dtype == CSK_F64 ? 8 : 4;
    char* w = static_cast<char*>(ws);
    void* A = w + H.A;
    void* b = w + H.b;
    void* x0 = x0_host ? w + H.x0 : nullptr;
    void* xs = x_star_host ? w + H.xs : nullptr;
    void* x = w + H.x;
    csk_info* info = reinterpret_cast<csk_info*>(w + H.info);
    CSK_CUDA_TRY(copy_in(A_host, m, n, lda, b_host, x0_host, x_star_host, s, A, b, x0, xs, st));
    rc = solve_enqueue(A, m, n, n, b, dtype, params, x0, xs, x, info, w + H.total, L, st);
    if (rc != CSK_OK) return rc;
    CSK_CUDA_TRY(cudaMemcpyAsync(x_out_host, x, (size_t)n * s, cudaMemcpyDeviceToHost, st));
    CSK_CUDA_TRY(cudaMemcpyAsync(info_host, info, sizeof(csk_info), cudaMemcpyDeviceToHost, st));
    CSK_CUDA_TRY(cudaStreamSynchronize(st));
    return info_host->status;
}

size_t csk_solve_host_many_workspace_size(const csk_host_problem* probs, int32_t count,
                                          int32_t dtype, const csk_params* params) {
    if (!probs || count < 1 || !params) return 0;
    size_t stage = 0, inner = 0;
    for (int32_t k = 0; k < count; ++k) {
        const size_t i = csk_solve_workspace_size(probs[k].m, probs[k].n, dtype, params);
        if (i == 0) return 0;
        HostStaging H;
        host_staging(probs[k].m, probs[k].n, dtype, &H);
        stage = std::max(stage, H.total);
        inner = std::max(inner, i);
    }
    return 2 * stage + inner;
}

int csk_solve_host_many(const csk_host_problem* probs, int32_t count, int32_t dtype,
                        const csk_params* params, void* ws, size_t ws_bytes, void* stream) {
    if (count == 0) return CSK_OK;
    if (!probs || count < 0 || !params || !ws) return CSK_EINVAL;
    size_t stage = 0;
    for (int32_t k = 0; k < count; ++k) {
        const csk_host_problem& q = probs[k];
        if (!q.A || !q.b || !q.x_out || !q.info) return CSK_EINVAL;
        int rc = check_solve_args(q.m, q.n, q.lda, dtype, params, ws);
        if (rc != CSK_OK) return rc;
        HostStaging H;
        host_staging(q.m, q.n, dtype, &H);
        stage = std::max(stage, H.total);
    }
    if (ws_bytes < csk_solve_host_many_workspace_size(probs, count, dtype, params))
        return CSK_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    const size_t s = dtype == CSK_F64 ? 8 : 4;
    char* w = static_cast<char*>(ws);
    char* inner = w + 2 * stage;

    // copies of problem k+1 run on `cp` while problem k is solved on `st`;
    // staging area k % 2 is reused once the solve that read it has finished
    CopyRes res;
    cudaError_t e = acquire_copy_res(&res);
    if (e != cudaSuccess) return CSK_ECUDA;
    cudaStream_t cp = res.cp;
    cudaEvent_t* copied = res.copied;
    cudaEvent_t* freed = res.freed;
    int first_bad = CSK_OK;
    // the copy stream starts after the work already queued on `st`
    if (e == cudaSuccess) e = cudaEventRecord(freed[0], st);
    if (e == cudaSuccess) e = cudaEventRecord(freed[1], st);
    auto slot_at = [&](int32_t k, HostStaging* H) {
        host_staging(probs[k].m, probs[k].n, dtype, H);
        return w + (k & 1) * stage;
    };
    // results of problem k go back after the copies of k+1 are queued: a
    // copy into pageable host memory holds the host until it is done, and
    // must not hold back the next problem's input copies
    auto queue_out = [&](int32_t k) {
        HostStaging H;
        char* sw = slot_at(k, &H);
        cudaError_t r = cudaMemcpyAsync(probs[k].x_out, sw + H.x, (size_t)probs[k].n * s,
                                        cudaMemcpyDeviceToHost, st);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(probs[k].info, sw + H.info, sizeof(csk_info),
                                cudaMemcpyDeviceToHost, st);
        if (r == cudaSuccess) r = cudaEventRecord(freed[k & 1], st);
        return r;
    };
    int32_t solved = 0;
    for (int32_t k = 0; k < count && e == cudaSuccess; ++k) {
        const csk_host_problem& q = probs[k];
        const int slot = k & 1;
        HostStaging H;
        char* sw = slot_at(k, &H);
        void* A = sw + H.A;
        void* b = sw + H.b;
        void* x0 = q.x0 ? sw + H.x0 : nullptr;
        void* xs = q.x_star ? sw + H.xs : nullptr;
        csk_info* info = reinterpret_cast<csk_info*>(sw + H.info);
        e = cudaStreamWaitEvent(cp, freed[slot], 0);
        if (e == cudaSuccess) e = copy_in(q.A, q.m, q.n, q.lda, q.b, q.x0, q.x_star, s, A, b, x0, xs, cp);
        if (e == cudaSuccess) e = cudaEventRecord(copied[slot], cp);
        if (e == cudaSuccess && k > 0) e = queue_out(k - 1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, copied[slot], 0);
        if (e != cudaSuccess) break;
        SolveLayout L;
        solve_layout(q.m, q.n, dtype, params->d, resolve_path(params->path, dtype, params->d, q.n), &L);
        first_bad = solve_enqueue(A, q.m, q.n, q.n, b, dtype, params, x0, xs, sw + H.x, info, inner,
                                  L, st);
        if (first_bad != CSK_OK) break;
        solved = k + 1;
    }
    if (e == cudaSuccess && first_bad == CSK_OK && solved == count) e = queue_out(count - 1);
    // drain both streams before the copy stream and events go back to the pool
    const cudaError_t e1 = cudaStreamSynchronize(cp);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    release_copy_res(res);
    if (e != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess) return CSK_ECUDA;
    if (first_bad != CSK_OK) return first_bad;
    for (int32_t k = 0; k < count; ++k)
        if (probs[k].info->status != CSK_OK) return probs[k].info->status;
    return CSK_OK;
}

}  // extern "C"
