// Quaternion-parameterised tangent frames (the 2DGS surfel form) and their
// adjoint, one thread per surfel.
//
// q = (w, x, y, z), used after normalisation: R = R(q / |q|), t_u and t_v
// are its first two columns. The adjoint turns dL/dt_u, dL/dt_v into dL/dq
// through the columns' partial derivatives and the normalisation
// (dL/dq = (I - qh qh^T) dL/dqh / |q|, qh = q / |q|).
#include "common.cuh"

namespace psi {
namespace {

__global__ void __launch_bounds__(256) frames_kernel(const float4 *__restrict__ q, int64_t n, float *tu, float *tv)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = q[i];
    const float r = rsqrtf(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
    const float w = v.x * r, x = v.y * r, y = v.z * r, z = v.w * r;
    tu[3 * i] = 1.0f - 2.0f * (y * y + z * z);
    tu[3 * i + 1] = 2.0f * (x * y + w * z);
    tu[3 * i + 2] = 2.0f * (x * z - w * y);
    tv[3 * i] = 2.0f * (x * y - w * z);
    tv[3 * i + 1] = 1.0f - 2.0f * (x * x + z * z);
    tv[3 * i + 2] = 2.0f * (y * z + w * x);
}

__global__ void __launch_bounds__(256) frames_bwd_kernel(const float4 *__restrict__ q, int64_t n, const float *g_tu,
                                                         const float *g_tv, float4 *g_q)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = q[i];
    const float nq = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
    const float w = v.x / nq, x = v.y / nq, y = v.z / nq, z = v.w / nq;
    const float gu0 = g_tu ? g_tu[3 * i] : 0.f, gu1 = g_tu ? g_tu[3 * i + 1] : 0.f, gu2 = g_tu ? g_tu[3 * i + 2] : 0.f;
    const float gv0 = g_tv ? g_tv[3 * i] : 0.f, gv1 = g_tv ? g_tv[3 * i + 1] : 0.f, gv2 = g_tv ? g_tv[3 * i + 2] : 0.f;
    // dL/d(w, x, y, z) of the unit quaternion
    const float gw = gu1 * 2.f * z - gu2 * 2.f * y - gv0 * 2.f * z + gv2 * 2.f * x;
    const float gx = gu1 * 2.f * y + gu2 * 2.f * z + gv0 * 2.f * y - gv1 * 4.f * x + gv2 * 2.f * w;
    const float gy = -gu0 * 4.f * y + gu1 * 2.f * x - gu2 * 2.f * w + gv0 * 2.f * x + gv2 * 2.f * z;
    const float gz = -gu0 * 4.f * z + gu1 * 2.f * w + gu2 * 2.f * x - gv0 * 2.f * w - gv1 * 4.f * z + gv2 * 2.f * y;
    // through the normalisation
    const float pr = gw * w + gx * x + gy * y + gz * z;
    float4 o = g_q[i];
    o.x += (gw - pr * w) / nq;
    o.y += (gx - pr * x) / nq;
    o.z += (gy - pr * y) / nq;
    o.w += (gz - pr * z) / nq;
    g_q[i] = o;
}

} // namespace

cudaError_t launch_frames(const float *q, int64_t n, float *tu, float *tv, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    frames_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4 *>(q), n, tu, tv);
    return cudaGetLastError();
}

cudaError_t launch_frames_bwd(const float *q, int64_t n, const float *g_tu, const float *g_tv, float *g_q,
                              cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    frames_bwd_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const float4 *>(q), n, g_tu, g_tv, reinterpret_cast<float4 *>(g_q));
    return cudaGetLastError();
}

} // namespace psi
