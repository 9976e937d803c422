// Zeroing of the gradient buffers before an accumulating adjoint (no
// counterpart in the paper; a training step's "zero the gradients").
//
// One kernel for all of them: a grid of eight 256-thread CTAs per SM looping
// over the buffers, four 16-byte stores per thread per iteration.
#include "common.cuh"

namespace psi {
namespace {

constexpr int kFillThreads = 256;
constexpr int kFillCtasPerSm = 8;

struct FillParts {
    float *p[kFillMaxParts];
    int64_t n[kFillMaxParts]; // floats
    int count;
};

__global__ void __launch_bounds__(kFillThreads, kFillCtasPerSm) zero_parts_kernel(const __grid_constant__ FillParts parts)
{
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int k = 0; k < parts.count; ++k) {
        float *p = parts.p[k];
        const int64_t n = parts.n[k];
        // head up to the first 16-byte boundary, the 16-byte body, the tail
        const int64_t mis = static_cast<int64_t>((16 - (reinterpret_cast<uintptr_t>(p) & 15)) & 15) / 4;
        const int64_t head = mis < n ? mis : n;
        const int64_t body = (n - head) / 4;
        if (tid < head) p[tid] = 0.0f;
        float4 *q = reinterpret_cast<float4 *>(p + head);
        const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int64_t i = tid;
        for (; i + 3 * nthreads < body; i += 4 * nthreads) {
            q[i] = z;
            q[i + nthreads] = z;
            q[i + 2 * nthreads] = z;
            q[i + 3 * nthreads] = z;
        }
        for (; i < body; i += nthreads) q[i] = z;
        const int64_t t0 = head + 4 * body;
        if (tid < n - t0) p[t0 + tid] = 0.0f;
    }
}

} // namespace

cudaError_t launch_zero_parts(float *const *ptrs, const int64_t *counts, int n_parts, cudaStream_t st)
{
    FillParts parts{};
    for (int k = 0; k < n_parts && k < kFillMaxParts; ++k) {
        if (!ptrs[k] || counts[k] <= 0) continue;
        parts.p[parts.count] = ptrs[k];
        parts.n[parts.count] = counts[k];
        ++parts.count;
    }
    if (parts.count == 0) return cudaSuccess;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    zero_parts_kernel<<<static_cast<unsigned>(sms * kFillCtasPerSm), kFillThreads, 0, st>>>(parts);
    return cudaGetLastError();
}

} // namespace psi
