// synth.cu -- seeded Gaussian test systems generated on the device.
//
// Not part of the method: the serving harness and benchmarks need systems
// A x* = b that "arrive" with their data, and generating each one with
// separate library calls costs more host time than solving it.  Every entry
// is a pure function of (system seed, matrix, element index): a SplitMix64
// counter hash gives two 32-bit uniforms and Box-Muller one standard normal,
// so a system's data do not depend on which other systems are generated in
// the same call.  B = A X* is accumulated in FP32 over the columns in
// ascending order (one warp per row: each lane sums its columns, then a
// fixed butterfly), also independent of the rest of the call.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace csk {

namespace {

constexpr uint64_t kDomainA = 0x6A09E667F3BCC909ull;   // keeps A, X and the sketch apart
constexpr uint64_t kDomainX = 0xBB67AE8584CAA73Bull;
constexpr int kSynthChunk = 32;                        // systems per launch (parameter space)
constexpr int kMaxSynthRhs = 16;

struct SynthDesc {
    float* A;
    float* X;
    float* B;
    uint64_t seed;
    int64_t row0;      // first global row of this system in the launch
    int32_t m, n, nrhs;
};

struct SynthChunk {
    SynthDesc e[kSynthChunk];
    int count;
    int64_t rows;      // total rows of the chunk
};

__device__ __forceinline__ float normal_at(uint64_t key, uint64_t idx) {
    const uint64_t u = row_hash(key, idx);
    const float u1 = ((float)(uint32_t)(u >> 32) + 0.5f) * 2.3283064365386963e-10f;   // (0, 1)
    const float u2 = (float)(uint32_t)u * 2.3283064365386963e-10f;                   // [0, 1)
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// X* of every system of the chunk: one thread per element.
__global__ void k_synth_x(SynthChunk c) {
    for (int s = 0; s < c.count; ++s) {
        const SynthDesc& e = c.e[s];
        const int64_t total = (int64_t)e.n * e.nrhs;
        const uint64_t key = e.seed ^ kDomainX;
        for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x)
            e.X[t] = normal_at(key, (uint64_t)t);
    }
}

// Rows of A and B: one warp per row of the chunk (rows numbered across its
// systems).
__global__ void k_synth_rows(SynthChunk c) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < c.rows;
         g += nwarps) {
        int s = 0;
        while (s + 1 < c.count && c.e[s + 1].row0 <= g) ++s;
        const SynthDesc& e = c.e[s];
        const int64_t i = g - e.row0;
        const int n = e.n, R = e.nrhs;
        const uint64_t key = e.seed ^ kDomainA;
        float acc[kMaxSynthRhs];
#pragma unroll
        for (int r = 0; r < kMaxSynthRhs; ++r) acc[r] = 0.0f;
        for (int j = lane; j < n; j += 32) {
            const float a = normal_at(key, (uint64_t)(i * n + j));
            e.A[i * n + j] = a;
#pragma unroll
            for (int r = 0; r < kMaxSynthRhs; ++r)
                if (r < R) acc[r] = fmaf(a, e.X[(int64_t)j * R + r], acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kMaxSynthRhs; ++r) {
            float v = acc[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (r < R && lane == 0) e.B[i * R + r] = v;
        }
    }
}

}  // namespace

int synth_systems(const csk_synth_system* sys, int count, cudaStream_t st) {
    DevInfo di;
    if (dev_info(&di) != 0) return CSK_ECUDA;
    for (int first = 0; first < count; first += kSynthChunk) {
        SynthChunk c;
        c.count = std::min(kSynthChunk, count - first);
        int64_t rows = 0, xs = 0;
        for (int q = 0; q < c.count; ++q) {
            const csk_synth_system& y = sys[first + q];
            c.e[q] = SynthDesc{static_cast<float*>(y.A), static_cast<float*>(y.X),
                               static_cast<float*>(y.B), y.seed, rows, (int32_t)y.m, (int32_t)y.n,
                               y.nrhs};
            rows += y.m;
            xs = std::max<int64_t>(xs, y.n * (int64_t)y.nrhs);
        }
        c.rows = rows;
        const int xblocks = (int)std::min<int64_t>((xs + 255) / 256, di.sms * 4);
        k_synth_x<<<std::max(1, xblocks), 256, 0, st>>>(c);
        const int rblocks = (int)std::min<int64_t>((rows + 7) / 8, (int64_t)di.sms * 16);
        k_synth_rows<<<std::max(1, rblocks), 256, 0, st>>>(c);
        note_launches(2);
    }
    return cudaGetLastError() == cudaSuccess ? CSK_OK : CSK_ECUDA;
}

}  // namespace csk

extern "C" int csk_synth_systems(const csk_synth_system* sys, int32_t count, void* stream) {
    if (count == 0) return CSK_OK;
    if (!sys || count < 0) return CSK_EINVAL;
    for (int32_t q = 0; q < count; ++q) {
        const csk_synth_system& y = sys[q];
        if (!y.A || !y.X || !y.B || y.m < 1 || y.n < 1 || y.nrhs < 1 || y.nrhs > csk::kMaxSynthRhs)
            return CSK_EINVAL;
        if (y.m > INT32_MAX || y.n > INT32_MAX || y.m * y.n > ((int64_t)1 << 40)) return CSK_ENOMEM;
    }
    return csk::synth_systems(sys, count, static_cast<cudaStream_t>(stream));
}
