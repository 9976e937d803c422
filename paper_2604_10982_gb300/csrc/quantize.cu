// Storage form of the per-surfel feature table: BF16 (round to nearest even)
// or FP8-E4M3 with a per-channel scale (amax_c / 448, values q = RNE(f /
// scale) saturated to the finite range), accumulated in FP32 by the
// compositing kernels. Run once per map.
//
// FP8: a column-max pass (each thread keeps the running |f| maximum of four
// channels over a strided set of rows, merged per block in shared memory and
// across blocks with integer atomicMax on the float bits, which order like the
// values for non-negative floats), a finalise pass that turns the maxima into
// scales in place, and the conversion pass.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace psi {
namespace {

constexpr int kQThreads = 256;

__global__ void __launch_bounds__(kQThreads) bf16_kernel(const float4 *__restrict__ f, int64_t n8, uint4 *__restrict__ q)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n8;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float4 a = f[2 * i], b = f[2 * i + 1];
        const __nv_bfloat162 p0 = __floats2bfloat162_rn(a.x, a.y), p1 = __floats2bfloat162_rn(a.z, a.w);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(b.x, b.y), p3 = __floats2bfloat162_rn(b.z, b.w);
        q[i] = make_uint4(*reinterpret_cast<const uint32_t *>(&p0), *reinterpret_cast<const uint32_t *>(&p1),
                          *reinterpret_cast<const uint32_t *>(&p2), *reinterpret_cast<const uint32_t *>(&p3));
    }
}

// amax_bits[c] (zeroed by the caller) <- max over rows of |f[r, c]| as float bits
__global__ void __launch_bounds__(kQThreads) amax_kernel(const float4 *__restrict__ f, int64_t n, int dim,
                                                         unsigned int *__restrict__ amax_bits)
{
    __shared__ unsigned int sm[256];
    const int g = dim / 4;                  // float4 groups per row
    const int rows_per_iter = kQThreads / g; // rows covered by one block step
    const int c4 = threadIdx.x % g, rsub = threadIdx.x / g;
    for (int c = threadIdx.x; c < dim; c += kQThreads) sm[c] = 0u;
    __syncthreads();
    if (rsub < rows_per_iter) {
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
        for (int64_t r = static_cast<int64_t>(blockIdx.x) * rows_per_iter + rsub; r < n;
             r += static_cast<int64_t>(gridDim.x) * rows_per_iter) {
            const float4 v = f[r * g + c4];
            m0 = fmaxf(m0, fabsf(v.x));
            m1 = fmaxf(m1, fabsf(v.y));
            m2 = fmaxf(m2, fabsf(v.z));
            m3 = fmaxf(m3, fabsf(v.w));
        }
        atomicMax(&sm[4 * c4 + 0], __float_as_uint(m0));
        atomicMax(&sm[4 * c4 + 1], __float_as_uint(m1));
        atomicMax(&sm[4 * c4 + 2], __float_as_uint(m2));
        atomicMax(&sm[4 * c4 + 3], __float_as_uint(m3));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < dim; c += kQThreads) atomicMax(&amax_bits[c], sm[c]);
}

// in place: scale[c] = max(amax_c, 1e-30) / 448 (448 = largest finite E4M3)
__global__ void scale_kernel(float *scale, int dim)
{
    const int c = threadIdx.x;
    if (c < dim) scale[c] = __fdiv_rn(fmaxf(scale[c], 1e-30f), 448.0f);
}

__device__ __forceinline__ uint32_t fp8x4(float a, float b, float c, float d)
{
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return lo | (hi << 16);
}

// 16 values per thread: q = RNE_satfinite(f / scale[c])
__global__ void __launch_bounds__(kQThreads) fp8_kernel(const float4 *__restrict__ f, int64_t n16, int dim,
                                                        const float *__restrict__ scale, uint4 *__restrict__ q)
{
    const int g16 = dim / 16;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c0 = static_cast<int>(i % g16) * 16;
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = f[4 * i + k];
            const float4 s = *reinterpret_cast<const float4 *>(scale + c0 + 4 * k);
            w[k] = fp8x4(__fdiv_rn(v.x, s.x), __fdiv_rn(v.y, s.y), __fdiv_rn(v.z, s.z), __fdiv_rn(v.w, s.w));
        }
        q[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

unsigned grid_for(int64_t items)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (items + kQThreads - 1) / kQThreads;
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(sms) * 8)));
}

} // namespace

cudaError_t launch_quantize(const float *f, int64_t n, int dim, int dtype, void *q, float *scale, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int64_t total = n * dim;
    if (dtype == PSI_BF16) {
        bf16_kernel<<<grid_for(total / 8), kQThreads, 0, st>>>(reinterpret_cast<const float4 *>(f), total / 8,
                                                               static_cast<uint4 *>(q));
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(scale, 0, static_cast<size_t>(dim) * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const int rows_per_iter = kQThreads / (dim / 4);
    amax_kernel<<<grid_for(n * kQThreads / rows_per_iter), kQThreads, 0, st>>>(
        reinterpret_cast<const float4 *>(f), n, dim, reinterpret_cast<unsigned int *>(scale));
    scale_kernel<<<1, 256, 0, st>>>(scale, dim);
    fp8_kernel<<<grid_for(total / 16), kQThreads, 0, st>>>(reinterpret_cast<const float4 *>(f), total / 16, dim, scale,
                                                            static_cast<uint4 *>(q));
    return cudaGetLastError();
}

} // namespace psi
