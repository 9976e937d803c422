// Per-surfel instance labels (Sec. 4.1, Eqs. 4-7) on the tensor cores.
//
// For surfel g (feature f_g, centre p_g) and instance query q (feature f_q,
// spatial Gaussian N(mu_q, Sigma_q)):
//     S(q, g) = sigmoid(f_q^T f_g)                                   (Eq. 4)
//     D(q, g) = phi_q(p_g) / phi_q(mu_q)
//             = exp(-(p_g - mu_q)^T Sigma_q^-1 (p_g - mu_q) / 2)      (Eq. 5)
//     l(g)    = softmax over q of S D                            (Eqs. 6-7)
// The dot products f_q^T f_g run in the row-tile tcgen05 pipeline
// (rowgemm.cuh: 128 surfels per tile, the queries resident in shared
// memory, FP32 accumulation in TMEM). The epilogue keeps each surfel's row of
// dot products in registers and applies the sigmoid, the geometric factor
// and the softmax in FP32; the queries' centres and precision matrices
// (inverted from Sigma once per CTA) sit in shared memory. The label table
// [n, ld] is written in FP32 or BF16 with zero columns past n_q, so it can be
// rendered like a feature table (Eq. 8).
#include <cuda_bf16.h>

#include "rowgemm.cuh"

namespace psi {
namespace {

using namespace tc;

constexpr int kQP = 12; // floats per query in shared memory: mu (3), precision (6), pad

struct LabelEpi {
    static constexpr int kStages = 2; // two CTAs per SM: the softmax epilogue dominates
    int64_t n;
    int n_q;
    const float *centres; // [n, 3]
    const float *q_mu;    // [n_q, 3]
    const float *q_cov;   // [n_q, 6]: xx, xy, xz, yy, yz, zz
    void *labels;         // [n, ld]
    int ld;
    int out_bf16;

    struct Pre {
        float x, y, z;
    };

    // each query's centre and precision Sigma^-1 (adjugate over determinant)
    __device__ __forceinline__ void prepare(unsigned char *smem, int tid) const
    {
        float *s = reinterpret_cast<float *>(smem);
        for (int q = tid; q < n_q; q += kRowThreads) {
            const float a = q_cov[6 * q], b = q_cov[6 * q + 1], c = q_cov[6 * q + 2];
            const float d = q_cov[6 * q + 3], e = q_cov[6 * q + 4], f = q_cov[6 * q + 5];
            const float A11 = d * f - e * e, A12 = c * e - b * f, A13 = b * e - c * d;
            const float A22 = a * f - c * c, A23 = b * c - a * e, A33 = a * d - b * b;
            const float inv = 1.0f / (a * A11 + b * A12 + c * A13);
            float *o = s + kQP * q;
            o[0] = q_mu[3 * q];
            o[1] = q_mu[3 * q + 1];
            o[2] = q_mu[3 * q + 2];
            o[3] = A11 * inv;
            o[4] = A12 * inv;
            o[5] = A13 * inv;
            o[6] = A22 * inv;
            o[7] = A23 * inv;
            o[8] = A33 * inv;
        }
    }

    __device__ __forceinline__ Pre begin(int64_t g) const
    {
        if (g >= n) return Pre{0.f, 0.f, 0.f};
        return Pre{__ldg(centres + 3 * g), __ldg(centres + 3 * g + 1), __ldg(centres + 3 * g + 2)};
    }

    // scores are computed in place over the row of dot products (r)
    __device__ __forceinline__ void end(int64_t g, uint32_t (&r)[kRowAccStride], Pre p, bool fail,
                                        unsigned char *smem) const
    {
        if (g >= n || fail) return;
        const float *s = reinterpret_cast<const float *>(smem);
        float *A = reinterpret_cast<float *>(r);
        float amax = -__int_as_float(0x7f800000);
#pragma unroll
        for (int q = 0; q < static_cast<int>(kRowAccStride); ++q) {
            if (q < n_q) {
                const float *o = s + kQP * q;
                const float dx = p.x - o[0], dy = p.y - o[1], dz = p.z - o[2];
                const float m2 = o[3] * dx * dx + o[6] * dy * dy + o[8] * dz * dz +
                                 2.0f * (o[4] * dx * dy + o[5] * dx * dz + o[7] * dy * dz);
                const float S = 1.0f / (1.0f + __expf(-A[q]));
                A[q] = S * __expf(-0.5f * m2);
                amax = fmaxf(amax, A[q]);
            }
        }
        float sum = 0.0f;
#pragma unroll
        for (int q = 0; q < static_cast<int>(kRowAccStride); ++q)
            if (q < n_q) {
                A[q] = __expf(A[q] - amax);
                sum += A[q];
            }
        const float inv = 1.0f / sum;
        // ld <= 128: every index below is a compile-time register
        if (out_bf16) {
            __nv_bfloat162 *row = reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(labels) + g * ld);
#pragma unroll
            for (int q = 0; q < static_cast<int>(kRowAccStride); q += 2)
                if (q < ld)
                    row[q >> 1] = __floats2bfloat162_rn(q < n_q ? A[q] * inv : 0.0f, q + 1 < n_q ? A[q + 1] * inv : 0.0f);
        } else {
            float4 *row = reinterpret_cast<float4 *>(static_cast<float *>(labels) + g * ld);
#pragma unroll
            for (int q = 0; q < static_cast<int>(kRowAccStride); q += 4)
                if (q < ld)
                    row[q >> 2] = make_float4(q < n_q ? A[q] * inv : 0.0f, q + 1 < n_q ? A[q + 1] * inv : 0.0f,
                                              q + 2 < n_q ? A[q + 2] * inv : 0.0f, q + 3 < n_q ? A[q + 3] * inv : 0.0f);
        }
    }
};

// The plain per-surfel query logits f_q^T f_g (no sigmoid, geometric factor
// or softmax): composited with the Top-K weights they give, by linearity,
// the decode's logits <F, q> of every pixel without forming F.
struct LogitEpi {
    static constexpr int kStages = 4; // one CTA per SM: bound by the table's stores
    int64_t n;
    int n_q;
    void *table; // [n, ld]
    int ld;
    int out_bf16;

    struct Pre {};
    __device__ __forceinline__ void prepare(unsigned char *, int) const {}
    __device__ __forceinline__ Pre begin(int64_t) const { return Pre{}; }
    __device__ __forceinline__ void end(int64_t g, uint32_t (&r)[kRowAccStride], Pre, bool fail, unsigned char *) const
    {
        if (g >= n || fail) return;
        const float *A = reinterpret_cast<const float *>(r);
        if (out_bf16) {
            __nv_bfloat162 *row = reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(table) + g * ld);
#pragma unroll
            for (int q = 0; q < static_cast<int>(kRowAccStride); q += 2)
                if (q < ld) row[q >> 1] = __floats2bfloat162_rn(q < n_q ? A[q] : 0.0f, q + 1 < n_q ? A[q + 1] : 0.0f);
        } else {
            float4 *row = reinterpret_cast<float4 *>(static_cast<float *>(table) + g * ld);
#pragma unroll
            for (int q = 0; q < static_cast<int>(kRowAccStride); q += 4)
                if (q < ld)
                    row[q >> 2] = make_float4(q < n_q ? A[q] : 0.0f, q + 1 < n_q ? A[q + 1] : 0.0f,
                                              q + 2 < n_q ? A[q + 2] : 0.0f, q + 3 < n_q ? A[q + 3] : 0.0f);
        }
    }
};

} // namespace

cudaError_t launch_logits(const void *F, int64_t n, int D, const void *Q, int n_q, void *table, int ld, int out_bf16,
                          DevStatus *status, cudaStream_t st, const char **why)
{
    const LogitEpi epi{n, n_q, table, ld, out_bf16};
    return launch_row_gemm(F, n, D, Q, n_q, 0, epi, status, st, why);
}

cudaError_t launch_labels(const void *F, int64_t n, int D, const float *centres, const void *Q, int n_q,
                          const float *q_mu, const float *q_cov, void *labels, int ld, int out_bf16, DevStatus *status,
                          cudaStream_t st, const char **why)
{
    const LabelEpi epi{n, n_q, centres, q_mu, q_cov, labels, ld, out_bf16};
    return launch_row_gemm(F, n, D, Q, n_q, static_cast<size_t>(kQP) * 128 * sizeof(float), epi, status, st, why);
}

} // namespace psi
