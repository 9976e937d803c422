// Frustum-constrained cross-attention (Sec. 4.1), forward.
//
// For the surfels j whose 99 % confidence disc meets the view frustum (the
// disc's bounding sphere, radius sqrt(chi2_2(0.99)) max(s_u, s_v), against
// the near plane and the four side planes of the image rectangle):
//     K_j = f_j + psi(mu_j),  V_j = f_j
//     e_ij = (Q_i W_Q)(K_j W_K)^T / sqrt(d),  Q'_i = softmax_j(e_ij) (V_j W_V)
// psi: channel c encodes axis c mod 3 with sin (t = c / 3 even) or cos (t odd)
// at frequency 10000^(-6k/C), k = t / 2.
// Backward (L = <G, Q'>): dP = G v^T, dv = P^T G, dE = P (dP - rowsum(P dP))
// / sqrt(d), dq = dE k, dk = dE^T q, and the projections' gradients; dK and
// dV land on the surfels' feature gradient and dK, through psi, on mu.
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

// row-major C[m x n] = A[m x k] B[n x k]^T
cublasStatus_t gemm_nt(cublasHandle_t h, int m, int n, int k, const float *A, const float *B, float *C)
{
    const float one = 1.0f, zero = 0.0f;
    return cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, n, m, k, &one, B, k, A, k, &zero, C, n);
}

// row-major C[m x n] = A[k x m]^T B[k x n]
cublasStatus_t gemm_tn(cublasHandle_t h, int m, int n, int k, const float *A, const float *B, float *C)
{
    const float one = 1.0f, zero = 0.0f;
    return cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, n, m, k, &one, B, n, A, m, &zero, C, n);
}

// One CTA per query row: dE = P (dP - sum_j P dP) * scale, in place over dP.
__global__ void __launch_bounds__(1024) attn_softmax_bwd_kernel(const float *P, float *dP, int64_t N, float scale)
{
    const float *p = P + static_cast<int64_t>(blockIdx.x) * N;
    float *g = dP + static_cast<int64_t>(blockIdx.x) * N;
    __shared__ float red[32];
    float s = 0.0f;
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) s += p[j] * g[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float x = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0) red[0] = x;
    }
    __syncthreads();
    const float rs = red[0];
    for (int64_t j = threadIdx.x; j < N; j += blockDim.x) g[j] = p[j] * (g[j] - rs) * scale;
}

// One warp per active surfel: feature gradient dK + dV, centre gradient
// sum_c dK_c dpsi_c/dmu (added to the gradient buffers).
__global__ void __launch_bounds__(256) attn_scatter_kernel(const float *dK, const float *dV, const uint8_t *active,
                                                           const float *mu, int64_t n, int C, float *g_feat,
                                                           float *g_mu)
{
    const int64_t j = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n || !active[j]) return;
    float gm[3] = {0.f, 0.f, 0.f};
    const float m[3] = {mu[3 * j], mu[3 * j + 1], mu[3 * j + 2]};
    const float lnb = 9.21034037198f; // ln 10000
    for (int c = lane; c < C; c += 32) {
        const float k = dK[j * C + c];
        if (g_feat) g_feat[j * C + c] += k + dV[j * C + c];
        const int t = c / 3, axis = c - 3 * t;
        const float w = __expf(-lnb * 6.0f * static_cast<float>(t >> 1) / static_cast<float>(C));
        const float arg = m[axis] * w;
        const float dpsi = ((t & 1) ? -sinf(arg) : cosf(arg)) * w;
        gm[axis] += k * dpsi;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gm[a] += __shfl_xor_sync(0xffffffffu, gm[a], o);
    if (lane == 0 && g_mu) {
        g_mu[3 * j] += gm[0];
        g_mu[3 * j + 1] += gm[1];
        g_mu[3 * j + 2] += gm[2];
    }
}

} // namespace

// forward: K, V [N, C]; k, v [N, d]; q [n_q, d]; S -> P [n_q, N]; mask [N];
// backward scratch: dP -> dE [n_q, N]; dq [n_q, d]; dk, dv [N, d]
size_t attention_workspace_bytes(int64_t n, int C, int d, int n_q)
{
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t N = static_cast<size_t>(std::max<int64_t>(n, 1));
    const size_t fwd = up(N * C * 4) * 2 + up(N * d * 4) * 2 + up(static_cast<size_t>(n_q) * d * 4) +
                       up(static_cast<size_t>(n_q) * N * 4) + up(N);
    return fwd + up(static_cast<size_t>(n_q) * N * 4) + up(static_cast<size_t>(n_q) * d * 4) + up(N * d * 4) * 2;
}

namespace {
struct AttnWs {
    float *K, *V, *k, *v, *q, *S, *dP, *dq, *dk, *dv;
    uint8_t *active;
};
AttnWs carve(void *ws, int64_t N, int C, int d, int n_q)
{
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += up(bytes);
        return r;
    };
    AttnWs w;
    w.K = reinterpret_cast<float *>(take(static_cast<size_t>(N) * C * 4));
    w.V = reinterpret_cast<float *>(take(static_cast<size_t>(N) * C * 4));
    w.k = reinterpret_cast<float *>(take(static_cast<size_t>(N) * d * 4));
    w.v = reinterpret_cast<float *>(take(static_cast<size_t>(N) * d * 4));
    w.q = reinterpret_cast<float *>(take(static_cast<size_t>(n_q) * d * 4));
    w.S = reinterpret_cast<float *>(take(static_cast<size_t>(n_q) * N * 4));
    w.active = reinterpret_cast<uint8_t *>(take(static_cast<size_t>(N)));
    w.dP = reinterpret_cast<float *>(take(static_cast<size_t>(n_q) * N * 4));
    w.dq = reinterpret_cast<float *>(take(static_cast<size_t>(n_q) * d * 4));
    w.dk = reinterpret_cast<float *>(take(static_cast<size_t>(N) * d * 4));
    w.dv = reinterpret_cast<float *>(take(static_cast<size_t>(N) * d * 4));
    return w;
}
} // namespace

cudaError_t launch_attention(void *cublas, const psi_surfels &s, const void *feat, const float *fscale, int dtype, int C,
                             const psi_camera &cam, float z_near, const float *Q, int n_q, const float *WQ,
                             const float *WK, const float *WV, int d, float *out, void *ws, cudaStream_t st,
                             const char **why)
{
    const int64_t N = s.n;
    const AttnWs w = carve(ws, N, C, d, n_q);
    float *K = w.K, *V = w.V, *k = w.k, *v = w.v, *q = w.q, *S = w.S;
    uint8_t *active = w.active;

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

cudaError_t launch_attention_bwd(void *cublas, int64_t N, int C, int n_q, const float *Q, const float *WQ,
                                 const float *WK, const float *WV, int d, const float *G, float *gQ, float *gWQ,
                                 float *gWK, float *gWV, const float *mu, float *g_feat, float *g_mu, void *ws,
                                 cudaStream_t st, const char **why)
{
    const AttnWs w = carve(ws, N, C, d, n_q);
    cublasHandle_t h = static_cast<cublasHandle_t>(cublas);
    const int n = static_cast<int>(N);
    auto ok = [&](cublasStatus_t s) { return s == CUBLAS_STATUS_SUCCESS; };
    if (!ok(cublasSetStream(h, st)) || !ok(gemm_nt(h, n_q, n, d, G, w.v, w.dP)) ||  // dP = G v^T
        !ok(gemm_tn(h, n, d, n_q, w.S, G, w.dv))) {                              // dv = P^T G
        *why = "cuBLAS GEMM failed";
        return cudaErrorUnknown;
    }
    attn_softmax_bwd_kernel<<<static_cast<unsigned>(n_q), 1024, 0, st>>>(w.S, w.dP, N,
                                                                         1.0f / sqrtf(static_cast<float>(d)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!ok(gemm_rm(h, n_q, d, n, w.dP, w.k, w.dq)) ||          // dq = dE k
        !ok(gemm_tn(h, n, d, n_q, w.dP, w.q, w.dk)) ||          // dk = dE^T q
        (gQ && !ok(gemm_nt(h, n_q, C, d, w.dq, WQ, gQ))) ||     // dQ = dq W_Q^T
        (gWQ && !ok(gemm_tn(h, C, d, n_q, Q, w.dq, gWQ))) ||    // dW_Q = Q^T dq
        (gWK && !ok(gemm_tn(h, C, d, n, w.K, w.dk, gWK))) ||    // dW_K = K^T dk
        (gWV && !ok(gemm_tn(h, C, d, n, w.V, w.dv, gWV))) ||    // dW_V = V^T dv
        !ok(gemm_nt(h, n, C, d, w.dk, WK, w.K)) ||              // dK = dk W_K^T (over K)
        !ok(gemm_nt(h, n, C, d, w.dv, WV, w.V))) {              // dV = dv W_V^T (over V)
        *why = "cuBLAS GEMM failed";
        return cudaErrorUnknown;
    }
    if (g_feat || g_mu)
        attn_scatter_kernel<<<static_cast<unsigned>((N * 32 + 255) / 256), 256, 0, st>>>(w.K, w.V, w.active, mu, N,
                                                                                         C, g_feat, g_mu);
    return cudaGetLastError();
}

} // namespace psi
