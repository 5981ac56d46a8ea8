// noalloc.cu -- csk_sketch_noalloc: the sketch entry point for callers that
// cannot allocate device memory.
//
// csk_sketch needs scratch for its counting sort (bucket counts, offsets and
// two row permutations) and asks the caller for it as a workspace.  Some
// callers have no way to provide one: code that is handed only input and
// output pointers by a host application that owns all device memory (a
// plugin or callback with no allocator in its interface), or latency-critical
// code that must not call cudaMalloc because it can synchronise the device
// and take driver-wide locks.  For them this file keeps the scratch in one
// statically sized device array that exists in every process that loads the
// library, on every GPU it touches, until the process exits.
#include <climits>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace csk {

namespace {

constexpr int64_t kNoAllocMaxRows = 1 << 20;      // m  <= 1,048,576
constexpr int64_t kNoAllocMaxBuckets = 1 << 18;   // d  <=   262,144

// Same carving as carve_sort_scratch() for the maximum sizes (a call that
// needs more is refused with CSK_ENOMEM, and a test runs the maximum sizes).
constexpr int64_t kScanTileRows = 4096;
constexpr int64_t kNoAllocBytes =
    ((kNoAllocMaxBuckets + 1) * 4 + 255) / 256 * 256 +           // cnt (+ claim counter)
    ((kNoAllocMaxBuckets + 1) * 4 + 255) / 256 * 256 +           // off
    2 * ((kNoAllocMaxRows * 4 + 255) / 256 * 256) +              // perm_tmp, perm
    (((kNoAllocMaxBuckets + kScanTileRows - 1) / kScanTileRows) * 4 + 255) / 256 * 256;

// The shared scratch.  In host code this name is only a stand-in for the
// device array; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];        // per device; set once its lookup succeeded

// Device address of the scratch on the current device.  The first call on a
// device looks it up (the one-time set-up) and keeps it for the life of the
// process; a failed lookup is not kept, so a later call tries again.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace csk

using namespace csk;

extern "C" int csk_sketch_noalloc(const void* A, int64_t m, int64_t n, int64_t lda,
                                  const void* B, int64_t ldb, int32_t nrhs, int32_t dtype,
                                  int64_t d, uint64_t seed, void* At, void* Bt,
                                  double* norms2_out, int32_t* perm_out, int32_t* off_out,
                                  void* stream) {
    if (!A || !At) return CSK_EINVAL;
    if (m < 1 || n < 1 || d < 1 || lda < n || nrhs < 0) return CSK_EINVAL;
    if (dtype != CSK_F32 && dtype != CSK_F64) return CSK_EINVAL;
    if (nrhs > 0 && (!B || !Bt || ldb < nrhs)) return CSK_EINVAL;
    if (m > kNoAllocMaxRows || d > kNoAllocMaxBuckets || n > INT_MAX) return CSK_ENOMEM;
    if ((int64_t)sort_scratch_bytes(m, d) > kNoAllocBytes) return CSK_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int rc = check_stream_device(st);
    if (rc != CSK_OK) return rc;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess || base == nullptr) return CSK_ECUDA;
    SortScratch s;
    carve_sort_scratch(base, m, d, &s);       // bucket counts are zeroed by the sort itself
    if (perm_out) s.perm = perm_out;
    if (off_out) s.off = off_out;
    if (launch_sketch(dtype, A, lda, m, (int)n, nrhs > 0 ? B : nullptr, ldb, nrhs, s, (int)d, seed,
                      At, Bt, norms2_out, st) != cudaSuccess)
        return CSK_ECUDA;
    return CSK_OK;
}
