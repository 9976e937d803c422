// Geometric and anisotropy regularisers of the joint objective (Sec. 4.2),
// fused into one pass over the surfels.
//
// For surfel i with an assigned planar prior k (centre m_k, unit normal
// nhat_k; k < 0: none):
//     L_geo = sum_i |(mu_i - m_k) . nhat_k| + lambda_n (1 - |n_i . nhat_k|),
//             n_i = c_i / |c_i|, c_i = t_u x t_v (the surfel normal)
//     L_iso = sum_i (s_i1 - s_i2)^2
// One thread per surfel computes both terms and the gradients of
// w_geo L_geo + w_iso L_iso, added to the gradient buffers (mu, t_u, t_v,
// s); the loss sums are reduced per block and added in float64.
#include "common.cuh"

namespace psi {
namespace {

struct RegArgs {
    psi_surfels s;
    const int32_t *node_of;
    const float *node_mu;
    const float *node_n;
    int64_t n_nodes;
    float lambda_n, w_geo, w_iso;
    double *losses; // [2]
    psi_grads g;
    DevStatus *status;
};

__device__ __forceinline__ float sgnf(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

__global__ void __launch_bounds__(256) regulariser_kernel(RegArgs a)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    double geo = 0.0, iso = 0.0;
    if (i < a.s.n) {
        // anisotropy
        const float s1 = a.s.scale[2 * i], s2 = a.s.scale[2 * i + 1];
        const float diff = s1 - s2;
        iso = static_cast<double>(diff) * diff;
        if (a.g.scale) {
            atomicAdd(a.g.scale + 2 * i, a.w_iso * 2.0f * diff);
            atomicAdd(a.g.scale + 2 * i + 1, -a.w_iso * 2.0f * diff);
        }
        // geometric prior
        const int k = a.node_of ? a.node_of[i] : -1;
        if (k >= a.n_nodes) {
            raise_status(a.status, PSI_ERR_INVALID_ARG);
        } else if (k >= 0) {
            const float3 mu = make_float3(a.s.mu[3 * i], a.s.mu[3 * i + 1], a.s.mu[3 * i + 2]);
            const float3 tu = make_float3(a.s.tu[3 * i], a.s.tu[3 * i + 1], a.s.tu[3 * i + 2]);
            const float3 tv = make_float3(a.s.tv[3 * i], a.s.tv[3 * i + 1], a.s.tv[3 * i + 2]);
            const float3 m = make_float3(a.node_mu[3 * k], a.node_mu[3 * k + 1], a.node_mu[3 * k + 2]);
            const float3 nh = make_float3(a.node_n[3 * k], a.node_n[3 * k + 1], a.node_n[3 * k + 2]);
            const float off = (mu.x - m.x) * nh.x + (mu.y - m.y) * nh.y + (mu.z - m.z) * nh.z;
            const float3 c = make_float3(tu.y * tv.z - tu.z * tv.y, tu.z * tv.x - tu.x * tv.z, tu.x * tv.y - tu.y * tv.x);
            const float cn = sqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
            const float3 n = make_float3(c.x / cn, c.y / cn, c.z / cn);
            const float dot = n.x * nh.x + n.y * nh.y + n.z * nh.z;
            geo = static_cast<double>(fabsf(off)) + static_cast<double>(a.lambda_n) * (1.0 - fabs(static_cast<double>(dot)));
            if (a.g.mu) {
                const float gm = a.w_geo * sgnf(off);
                atomicAdd(a.g.mu + 3 * i, gm * nh.x);
                atomicAdd(a.g.mu + 3 * i + 1, gm * nh.y);
                atomicAdd(a.g.mu + 3 * i + 2, gm * nh.z);
            }
            // dL/dn = -lambda_n sign(n.nhat) nhat; dL/dc = (I - n n^T) dL/dn / |c|
            const float gs = -a.w_geo * a.lambda_n * sgnf(dot);
            const float3 gn = make_float3(gs * nh.x, gs * nh.y, gs * nh.z);
            const float pr = gn.x * n.x + gn.y * n.y + gn.z * n.z;
            const float3 gc = make_float3((gn.x - pr * n.x) / cn, (gn.y - pr * n.y) / cn, (gn.z - pr * n.z) / cn);
            if (a.g.tu) { // dL/dtu = tv x dL/dc
                atomicAdd(a.g.tu + 3 * i, tv.y * gc.z - tv.z * gc.y);
                atomicAdd(a.g.tu + 3 * i + 1, tv.z * gc.x - tv.x * gc.z);
                atomicAdd(a.g.tu + 3 * i + 2, tv.x * gc.y - tv.y * gc.x);
            }
            if (a.g.tv) { // dL/dtv = dL/dc x tu
                atomicAdd(a.g.tv + 3 * i, gc.y * tu.z - gc.z * tu.y);
                atomicAdd(a.g.tv + 3 * i + 1, gc.z * tu.x - gc.x * tu.z);
                atomicAdd(a.g.tv + 3 * i + 2, gc.x * tu.y - gc.y * tu.x);
            }
        }
    }
    // block sums of the two losses (warp shuffles, then one lane per warp)
    __shared__ double part[2][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        geo += __shfl_xor_sync(0xffffffffu, geo, o);
        iso += __shfl_xor_sync(0xffffffffu, iso, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        part[0][w] = geo;
        part[1][w] = iso;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double g0 = 0.0, g1 = 0.0;
        for (int k = 0; k < (blockDim.x >> 5); ++k) {
            g0 += part[0][k];
            g1 += part[1][k];
        }
        atomicAdd(a.losses, g0);
        atomicAdd(a.losses + 1, g1);
    }
}

} // namespace

cudaError_t launch_regularisers(const psi_surfels &s, const int32_t *node_of, const float *node_mu, const float *node_n,
                                int64_t n_nodes, float lambda_n, float w_geo, float w_iso, double *losses,
                                const psi_grads &g, DevStatus *status, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(losses, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess || s.n == 0) return e;
    RegArgs a{s, node_of, node_mu, node_n, n_nodes, lambda_n, w_geo, w_iso, losses, g, status};
    regulariser_kernel<<<static_cast<unsigned>((s.n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

} // namespace psi
