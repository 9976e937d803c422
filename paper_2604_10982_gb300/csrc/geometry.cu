// Per-surfel geometry table for depth and normal maps of the 2D-surfel model
// (Sec. 3.1), and its adjoint.
//
// For surfel i and one camera: z_i = (R mu_i + t)_z, the camera depth of the
// centre, and n_i = R (t_u x t_v) / |t_u x t_v|, the unit normal in camera
// coordinates turned to face the camera (negated where n . x_c > 0). The
// table row is (z, n_x, n_y, n_z, 0, ...) with ld floats, so the dense
// (K = 0) feature path of the compositing kernel blends it into the expected
// depth sum_j omega_j z_j and normal sum_j omega_j n_j maps; the adjoint of
// that render gives dL/dtable (its feature gradient), which the second kernel
// takes to mu, t_u and t_v. One thread per surfel.
#include "geometry.cuh"

namespace psi {
namespace {

struct GeoCam {
    float R[9];
    float t[3];
};

__device__ __forceinline__ void frame_of(const psi_surfels &s, int64_t i, const GeoCam &c, float xc[3], float nw[3],
                                          float &cn, bool &flip)
{
    const float m0 = s.mu[3 * i], m1 = s.mu[3 * i + 1], m2 = s.mu[3 * i + 2];
    for (int k = 0; k < 3; ++k) xc[k] = c.R[3 * k] * m0 + c.R[3 * k + 1] * m1 + c.R[3 * k + 2] * m2 + c.t[k];
    const float u0 = s.tu[3 * i], u1 = s.tu[3 * i + 1], u2 = s.tu[3 * i + 2];
    const float v0 = s.tv[3 * i], v1 = s.tv[3 * i + 1], v2 = s.tv[3 * i + 2];
    const float c0 = u1 * v2 - u2 * v1, c1 = u2 * v0 - u0 * v2, c2 = u0 * v1 - u1 * v0;
    cn = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
    nw[0] = c0 / cn;
    nw[1] = c1 / cn;
    nw[2] = c2 / cn;
    float dot = 0.0f;
    for (int k = 0; k < 3; ++k) dot += (c.R[3 * k] * nw[0] + c.R[3 * k + 1] * nw[1] + c.R[3 * k + 2] * nw[2]) * xc[k];
    flip = dot > 0.0f;
}

__global__ void __launch_bounds__(256) geometry_kernel(psi_surfels s, GeoCam c, float *__restrict__ table, int ld)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    float xc[3], nw[3], cn;
    bool flip;
    frame_of(s, i, c, xc, nw, cn, flip);
    const float sg = flip ? -1.0f : 1.0f;
    float *row = table + i * ld;
    float4 *row4 = reinterpret_cast<float4 *>(row);
    row4[0] = make_float4(xc[2], sg * (c.R[0] * nw[0] + c.R[1] * nw[1] + c.R[2] * nw[2]),
                          sg * (c.R[3] * nw[0] + c.R[4] * nw[1] + c.R[5] * nw[2]),
                          sg * (c.R[6] * nw[0] + c.R[7] * nw[1] + c.R[8] * nw[2]));
    for (int k = 1; k < ld / 4; ++k) row4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(256) geometry_bwd_kernel(psi_surfels s, GeoCam c, const float *__restrict__ g_table,
                                                           int ld, psi_grads g)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const float4 gr = reinterpret_cast<const float4 *>(g_table + i * ld)[0];
    if (gr.x == 0.0f && gr.y == 0.0f && gr.z == 0.0f && gr.w == 0.0f) return;
    float xc[3], nw[3], cn;
    bool flip;
    frame_of(s, i, c, xc, nw, cn, flip);
    // z = R[2] . mu + t_z
    if (g.mu)
        for (int k = 0; k < 3; ++k) atomicAdd(g.mu + 3 * i + k, gr.x * c.R[6 + k]);
    if (!g.tu && !g.tv) return;
    const float sg = flip ? -1.0f : 1.0f;
    const float gc_[3] = {sg * gr.y, sg * gr.z, sg * gr.w};
    float gw[3]; // n_c = R n_w: dL/dn_w = R^T dL/dn_c
    for (int k = 0; k < 3; ++k) gw[k] = c.R[k] * gc_[0] + c.R[3 + k] * gc_[1] + c.R[6 + k] * gc_[2];
    // n_w = c/|c|: dL/dc = (I - n n^T) dL/dn / |c|
    const float pr = gw[0] * nw[0] + gw[1] * nw[1] + gw[2] * nw[2];
    const float gcx = (gw[0] - pr * nw[0]) / cn, gcy = (gw[1] - pr * nw[1]) / cn, gcz = (gw[2] - pr * nw[2]) / cn;
    const float u0 = s.tu[3 * i], u1 = s.tu[3 * i + 1], u2 = s.tu[3 * i + 2];
    const float v0 = s.tv[3 * i], v1 = s.tv[3 * i + 1], v2 = s.tv[3 * i + 2];
    if (g.tu) { // c = t_u x t_v: dL/dt_u = t_v x dL/dc
        atomicAdd(g.tu + 3 * i, v1 * gcz - v2 * gcy);
        atomicAdd(g.tu + 3 * i + 1, v2 * gcx - v0 * gcz);
        atomicAdd(g.tu + 3 * i + 2, v0 * gcy - v1 * gcx);
    }
    if (g.tv) { // dL/dt_v = dL/dc x t_u
        atomicAdd(g.tv + 3 * i, gcy * u2 - gcz * u1);
        atomicAdd(g.tv + 3 * i + 1, gcz * u0 - gcx * u2);
        atomicAdd(g.tv + 3 * i + 2, gcx * u1 - gcy * u0);
    }
}

GeoCam geo_cam(const psi_camera &cam)
{
    GeoCam c;
    for (int k = 0; k < 9; ++k) c.R[k] = cam.R[k];
    for (int k = 0; k < 3; ++k) c.t[k] = cam.t[k];
    return c;
}

} // namespace

cudaError_t launch_geometry(const psi_surfels &s, const psi_camera &cam, float *table, int ld, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    geometry_kernel<<<static_cast<unsigned>((s.n + 255) / 256), 256, 0, st>>>(s, geo_cam(cam), table, ld);
    return cudaGetLastError();
}

cudaError_t launch_geometry_bwd(const psi_surfels &s, const psi_camera &cam, const float *g_table, int ld,
                                const psi_grads &g, cudaStream_t st)
{
    if (s.n == 0) return cudaSuccess;
    geometry_bwd_kernel<<<static_cast<unsigned>((s.n + 255) / 256), 256, 0, st>>>(s, geo_cam(cam), g_table, ld, g);
    return cudaGetLastError();
}

} // namespace psi
