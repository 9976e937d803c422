// Frustum-constrained cross-attention (Sec. 4.1), forward.
//
// For the surfels j whose 99 % confidence disc meets the view frustum (the
// disc's bounding sphere, radius sqrt(chi2_2(0.99)) max(s_u, s_v), against
// the near plane and the four side planes of the image rectangle):
//     K_j = f_j + psi(mu_j),  V_j = f_j
//     e_ij = (Q_i W_Q)(K_j W_K)^T / sqrt(d),  Q'_i = softmax_j(e_ij) (V_j W_V)
// psi: channel c encodes axis c mod 3 with sin (t = c / 3 even) or cos (t odd)
// at frequency 10000^(-6k/C), k = t / 2.
// A kernel builds K, V (float32 rows) and the active mask for every surfel;
// the four products run as FP32 cuBLAS GEMMs (plain library GEMMs) over all
// surfels; the row softmax masks inactive surfels (weight 0) and applies the
// 1/sqrt(d) scale. Masking instead of compacting keeps the call free of host
// synchronisation (and capturable in a CUDA graph).
#include <cublas_v2.h>

#include "common.cuh"

namespace psi {
namespace {

constexpr float kChi2_99 = 9.21034037198f; // -2 ln 0.01

struct AttnPrep {
    psi_surfels s;
    const void *feat;
    const float *fscale;
    int dtype;
    int C;
    float R[9], t[3], fx, fy, cx, cy, W, H, z_near;
    float *K;          // [N, C]
    float *V;          // [N, C]
    uint8_t *active;   // [N]
};

__device__ __forceinline__ float feat_value(const AttnPrep &a, int64_t j, int c)
{
    float v;
    if (a.dtype == PSI_F32) {
        v = static_cast<const float *>(a.feat)[j * a.C + c];
    } else if (a.dtype == PSI_BF16) {
        const uint16_t b = static_cast<const uint16_t *>(a.feat)[j * a.C + c];
        v = __uint_as_float(static_cast<uint32_t>(b) << 16);
    } else {
        const uint32_t byte = static_cast<const uint8_t *>(a.feat)[j * a.C + c];
        v = __uint_as_float(((byte & 0x80u) << 24) | ((byte & 0x7Fu) << 20)) * 0x1p120f;
    }
    return a.fscale ? v * a.fscale[c] : v;
}

// one warp per surfel: the mask, then the K and V rows with lanes across channels
__global__ void __launch_bounds__(256) attn_prep_kernel(const __grid_constant__ AttnPrep a)
{
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= a.s.n) return;
    const float mx = a.s.mu[3 * j], my = a.s.mu[3 * j + 1], mz = a.s.mu[3 * j + 2];
    if (lane == 0) {
        const float x = a.R[0] * mx + a.R[1] * my + a.R[2] * mz + a.t[0];
        const float y = a.R[3] * mx + a.R[4] * my + a.R[5] * mz + a.t[1];
        const float z = a.R[6] * mx + a.R[7] * my + a.R[8] * mz + a.t[2];
        const float r = sqrtf(kChi2_99) * fmaxf(a.s.scale[2 * j], a.s.scale[2 * j + 1]);
        float d = z - a.z_near;
        d = fminf(d, (a.fx * x + a.cx * z) * rsqrtf(a.fx * a.fx + a.cx * a.cx));
        d = fminf(d, (-a.fx * x + (a.W - a.cx) * z) * rsqrtf(a.fx * a.fx + (a.W - a.cx) * (a.W - a.cx)));
        d = fminf(d, (a.fy * y + a.cy * z) * rsqrtf(a.fy * a.fy + a.cy * a.cy));
        d = fminf(d, (-a.fy * y + (a.H - a.cy) * z) * rsqrtf(a.fy * a.fy + (a.H - a.cy) * (a.H - a.cy)));
        a.active[j] = d + r >= 0.0f ? 1 : 0;
    }
    const float lnb = 9.21034037198f; // ln 10000
    for (int c = lane; c < a.C; c += 32) {
        const int t = c / 3, axis = c - 3 * t, k = t >> 1;
        const float w = __expf(-lnb * 6.0f * static_cast<float>(k) / static_cast<float>(a.C));
        const float m = axis == 0 ? mx : (axis == 1 ? my : mz);
        const float pe = (t & 1) ? cosf(m * w) : sinf(m * w);
        const float f = feat_value(a, j, c);
        a.K[j * a.C + c] = f + pe;
        a.V[j * a.C + c] = f;
    }
}

// One CTA per query row of S [n_q, N] (scores): P = masked softmax(S / sqrt(d)),
// written in place; inactive surfels get weight 0.
__global__ void __launch_bounds__(1024) attn_softmax_kernel(float *S, int64_t N, const uint8_t *active, float scale)
{
    float *row = S + static_cast<int64_t>(blockIdx.x) * N;
    __shared__ float red[32];
    // pass 1: maximum over active entries
    float m = -__int_as_float(0x7f800000);
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x)
        if (active[j]) m = fmaxf(m, row[j] * scale);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -__int_as_float(0x7f800000);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (threadIdx.x == 0) red[0] = x;
    }
    __syncthreads();
    m = red[0];
    __syncthreads();
    // pass 2: exponentials and their sum
    float sum = 0.0f;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
        const float e = active[j] ? __expf(row[j] * scale - m) : 0.0f;
        row[j] = e;
        sum += e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x < 32) {
        float x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) red[0] = x;
    }
    __syncthreads();
    const float inv = red[0] > 0.0f ? 1.0f / red[0] : 0.0f;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) row[j] *= inv;
}

// row-major C[m x n] = A[m x k] B[k x n] (float32) with column-major cuBLAS
cublasStatus_t gemm_rm(cublasHandle_t h, int m, int n, int k, const float *A, const float *B, float *C)
{
    const float one = 1.0f, zero = 0.0f;
    return cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, n, m, k, &one, B, n, A, k, &zero, C, n);
}

} // namespace

size_t attention_workspace_bytes(int64_t n, int C, int d, int n_q)
{
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t N = static_cast<size_t>(std::max<int64_t>(n, 1));
    return up(N * C * 4) * 2 + up(N * d * 4) * 2 + up(static_cast<size_t>(n_q) * d * 4) +
           up(static_cast<size_t>(n_q) * N * 4) + up(N);
}

cudaError_t launch_attention(void *cublas, const psi_surfels &s, const void *feat, const float *fscale, int dtype, int C,
                             const psi_camera &cam, float z_near, const float *Q, int n_q, const float *WQ,
                             const float *WK, const float *WV, int d, float *out, void *ws, cudaStream_t st,
                             const char **why)
{
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const int64_t N = s.n;
    char *p = static_cast<char *>(ws);
    float *K = reinterpret_cast<float *>(p);
    p += up(static_cast<size_t>(N) * C * 4);
    float *V = reinterpret_cast<float *>(p);
    p += up(static_cast<size_t>(N) * C * 4);
    float *k = reinterpret_cast<float *>(p);
    p += up(static_cast<size_t>(N) * d * 4);
    float *v = reinterpret_cast<float *>(p);
    p += up(static_cast<size_t>(N) * d * 4);
    float *q = reinterpret_cast<float *>(p);
    p += up(static_cast<size_t>(n_q) * d * 4);
    float *S = reinterpret_cast<float *>(p);
    p += up(static_cast<size_t>(n_q) * N * 4);
    uint8_t *active = reinterpret_cast<uint8_t *>(p);

    AttnPrep a{};
    a.s = s;
    a.feat = feat;
    a.fscale = fscale;
    a.dtype = dtype;
    a.C = C;
    for (int i = 0; i < 9; ++i) a.R[i] = cam.R[i];
    for (int i = 0; i < 3; ++i) a.t[i] = cam.t[i];
    a.fx = cam.fx;
    a.fy = cam.fy;
    a.cx = cam.cx;
    a.cy = cam.cy;
    a.W = static_cast<float>(cam.width);
    a.H = static_cast<float>(cam.height);
    a.z_near = z_near;
    a.K = K;
    a.V = V;
    a.active = active;
    attn_prep_kernel<<<static_cast<unsigned>((N * 32 + 255) / 256), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cublasHandle_t h = static_cast<cublasHandle_t>(cublas);
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS ||
        gemm_rm(h, n_q, d, C, Q, WQ, q) != CUBLAS_STATUS_SUCCESS ||
        gemm_rm(h, static_cast<int>(N), d, C, K, WK, k) != CUBLAS_STATUS_SUCCESS ||
        gemm_rm(h, static_cast<int>(N), d, C, V, WV, v) != CUBLAS_STATUS_SUCCESS) {
        *why = "cuBLAS GEMM failed";
        return cudaErrorUnknown;
    }
    // S [n_q x N] = q [n_q x d] k^T: column-major S^T [N x n_q] = (k as [N x d]) q^T
    const float one = 1.0f, zero = 0.0f;
    if (cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, static_cast<int>(N), n_q, d, &one, k, d, q, d, &zero, S,
                    static_cast<int>(N)) != CUBLAS_STATUS_SUCCESS) {
        *why = "cuBLAS GEMM failed";
        return cudaErrorUnknown;
    }
    attn_softmax_kernel<<<static_cast<unsigned>(n_q), 1024, 0, st>>>(S, N, active, 1.0f / sqrtf(static_cast<float>(d)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // out [n_q x d] = P [n_q x N] v [N x d]
    if (gemm_rm(h, n_q, d, static_cast<int>(N), S, v, out) != CUBLAS_STATUS_SUCCESS) {
        *why = "cuBLAS GEMM failed";
        return cudaErrorUnknown;
    }
    return cudaSuccess;
}

} // namespace psi
