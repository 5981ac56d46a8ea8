// kernels.h -- host-side launchers of the CSK kernels (internal to libcsk).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "csk.h"

namespace csk {

// Device properties cached per device (SM count, shared memory limits).
struct DevInfo {
    int sms = 0;
    int smem_optin = 0;     // max dynamic shared memory per block (bytes)
    int smem_per_sm = 0;    // shared memory per multiprocessor (bytes)
    int coop = 0;           // cooperative launch supported
};
int dev_info(DevInfo* out);

// Kernel attributes and occupancy, set / queried once per (device, kernel,
// value) and cached: cudaFuncSetAttribute may not be called while a stream is
// being captured into a CUDA graph, so after a first (uncaptured) call the
// launch sequences make no such call.
cudaError_t ensure_smem_attr(const void* fn, size_t smem);
cudaError_t cached_occupancy(const void* fn, int threads, size_t smem, int* per_sm);

// Count of kernels enqueued by the library (csk_kernel_launches).
void note_launches(int k);

// CSK_OK when `st` is NULL or belongs to the current device (or is being
// captured, when its device cannot be queried), CSK_EINVAL otherwise.
int check_stream_device(cudaStream_t st);

// ------------------------------------------------------------- sketch
// Scratch of the counting sort: cnt[d + 1] (bucket counts, then the bucket
// claim counter of the segmented sum), off[d+1], perm_tmp[m], perm[m], scan
// partials.  All int32.
struct SortScratch {
    int32_t* cnt;
    int32_t* off;
    int32_t* perm_tmp;
    int32_t* perm;
    int32_t* part;
};
size_t sort_scratch_bytes(int64_t m, int64_t d);
void carve_sort_scratch(void* base, int64_t m, int64_t d, SortScratch* s);

// Rows grouped by bucket (hist -> scan -> scatter): off[d+1], and perm_tmp[m]
// holding each bucket's rows in no particular order.
cudaError_t launch_bucket_group(int64_t m, int64_t d, uint64_t seed, const SortScratch& s,
                                cudaStream_t st);

// Segmented signed row sum At = S A, Bt = S B (+ FP64 row norms), after
// launch_bucket_group; also writes perm[m], the rows sorted by (h(i), i).
cudaError_t launch_segsum(int dtype, const void* A, int64_t lda, int64_t m, int n, const void* B,
                          int64_t ldb, int nrhs, const SortScratch& s, int d, uint64_t seed,
                          void* At, void* Bt, double* N2, cudaStream_t st);

// The whole sketch: the counting-sort path (launch_bucket_group, then
// launch_segsum), or for FP32 sketches with small buckets the bucket-owner
// path (a hash pass and one kernel, no global sort).  Same outputs, same bits.
cudaError_t launch_sketch(int dtype, const void* A, int64_t lda, int64_t m, int n, const void* B,
                          int64_t ldb, int nrhs, const SortScratch& s, int d, uint64_t seed,
                          void* At, void* Bt, double* N2, cudaStream_t st);

// FP64 squared row norms of a (rows x n, ld) matrix (unsketched path).
cudaError_t launch_row_norms(int dtype, const void* A, int64_t ld, int rows, int n,
                             double* N2, cudaStream_t st);

// out[0] = sum_i v_i^2 in FP64 (one block, fixed order).
cudaError_t launch_norm2(int dtype, const void* v, int64_t len, double* out, cudaStream_t st);

// -------------------------------------------------------------- iterate
// Largest CTA count of the persistent loop; the exchange mailboxes take
// 2 * grid * grid slots of 64 bytes (FP32 rounds use the first half of the
// area, 32-byte slots; FP64 rounds all of it).
constexpr int kMaxIterGrid = 320;
inline size_t exchange_bytes(int grid) { return (size_t)2 * grid * grid * 64; }
struct IterConfig {
    int grid = 0;           // CTAs
    int threads = 256;
    int rows_per_cta = 0;
    int cache_rows = 0;     // At slice resident in shared memory (GEMV path)
    int reg_rpw = 0;        // >0: register-resident GEMV variant, rows per warp
    int reg_cpl = 0;        //     and float4 columns per lane
    int stream_cpl = 0;     // >0: rows streamed through a bulk-copy ring (FP32 GEMV)
    int stream_stages = 0;  //     and the ring's depth in blocks
    size_t smem = 0;        // dynamic shared memory bytes
};

struct IterProblem {
    int dtype;
    const void* At;  int64_t ld;  int d;  int n;
    const void* bt;  const double* N2;
    const void* x0;  const void* xstar;  void* x_out;
    const double* stop_norm;   // ||x*||^2, or ||bt||^2 without x*
    Slot* slots;               // 2 * grid
    void* xg;                  // n elements (GRAM path refresh)
    const float* G;  int64_t ldg;  // GRAM path
    int refresh_every;
    int32_t* ik_log;  int64_t ik_log_len;
    void* x_log;  int64_t x_log_len;
    double tol;  int64_t max_iter;  int64_t spin_limit;  int fault_inject;
    csk_info* info;
};

// variant: 0 = library choice, 1 = shared-memory rows, 2 = register rows.
// vec_ok: rows of At are 16-byte aligned with a leading dimension % 4 == 0.
int plan_iterate(int path, int dtype, int d, int n, int grid_req, int variant, bool vec_ok,
                 IterConfig* cfg);
cudaError_t launch_iterate(int path, const IterProblem& p, const IterConfig& cfg, cudaStream_t st);

// The fused sketch-and-loop launch (GEMV path, register or shared-memory
// loop, d <= 65535): the sketch of A is formed inside the loop's cooperative
// kernel, each CTA sketching the rows it then owns.  h / perm / off are sort
// scratch, part one double per CTA.
struct FusedArgs {
    const void* A;
    int64_t lda, m;
    const void* b;
    uint64_t seed;
    uint16_t* h;
    int32_t* perm;
    int32_t* off;
    double* part;
};
int plan_fused(int dtype, int64_t m, int d, int n, const IterConfig& cfg, const void* A,
               int64_t lda, int* cap, size_t* smem);
cudaError_t launch_fused(int dtype, const IterProblem& p, const IterConfig& cfg,
                         const FusedArgs& fa, int cap, size_t smem, cudaStream_t st);

// Exchange-only loop of `grid` CTAs for `rounds` rounds (csk_exchange_floor).
cudaError_t launch_exchange_probe(int grid, int64_t rounds, Slot* slots, csk_info* info,
                                  cudaStream_t st);

// FP64 final check: info->rse, info->resid, info->empty_rows.
cudaError_t launch_final_check(int dtype, const void* At, int64_t ld, int d, int n,
                               const void* bt, const double* N2, const void* x,
                               const void* xstar, double* partials, csk_info* info,
                               cudaStream_t st);
size_t final_check_partials(int d);

// -------------------------------------------------------------- batched
size_t batched_workspace_bytes(const csk_system* sys, int nsys, bool prepare, bool iterate);
size_t batched_area_bytes(int64_t n, int64_t d, int32_t nrhs);
// Per-step logs of one (system, right-hand side) pair: the caller's system
// index and column; ik / x may be NULL.
struct BatchLog {
    int system = -1, rhs = 0;
    int32_t* ik = nullptr;  int64_t ik_len = 0;
    float* x = nullptr;     int64_t x_len = 0;
};
// Tuned launch shape for batches of this signature (threads = grid = 0
// removes it); csk_solve_batched with threads = grid = 0 uses it.
int set_batched_plan(const csk_system* sys, int nsys, int threads, int grid);
uint64_t batched_signature(const csk_system* sys, int nsys);
int launch_batched(const csk_system* sys, int nsys, const csk_params* p, const BatchLog& log,
                   void* ws, size_t ws_bytes, cudaStream_t st);
int launch_batched_prepare(const csk_system* sys, int nsys, void* ws, size_t ws_bytes,
                           cudaStream_t st);
int launch_batched_iterate(const csk_system* sys, int nsys, const csk_params* p,
                           const BatchLog& log, int64_t budget, void* ws, size_t ws_bytes,
                           cudaStream_t st);

// ----------------------------------------------------------------- Gram
// G = At At^T (d x d, FP32) from split BF16 operands on the tensor cores;
// G_jj set to fl32(N2_j).
int64_t gram_ld(int d);   // leading dimension of G (multiple of 32)
size_t gram_scratch_bytes(int d, int n);
cudaError_t launch_gram_split_bf16(const float* At, int d, int n, const double* N2, float* G,
                                   int64_t ldg, void* scratch, csk_info* info, cudaStream_t st);

}  // namespace csk
