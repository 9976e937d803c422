// a6: query decode on the 5th-generation tensor cores.
//
// logits[p, q] = sum_c F[p, c] Q[q, c] (the feature similarity f_q^T f_g of
// Sec. 4.1, Eq. 4, before its monotone sigmoid), then the per-pixel argmax
// (lowest q on ties) as the panoptic id, -1 where nothing was rendered.
// The contraction runs in the row-tile tcgen05 pipeline of rowgemm.cuh
// (128 pixels per tile, Q resident in shared memory); the epilogue reduces
// each pixel's row of logits in registers.
#include <cuda_bf16.h>

#include "rowgemm.cuh"

namespace psi {
namespace {

using namespace tc;

struct DecodeEpi {
    static constexpr int kStages = 2; // two CTAs per SM: the per-row argmax dominates
    int64_t n_pix;
    int n_q;
    const float *T;
    int32_t *ids;
    __nv_bfloat16 *logits;

    struct Pre {
        float T;
    };
    __device__ __forceinline__ void prepare(unsigned char *, int) const {}
    __device__ __forceinline__ Pre begin(int64_t pix) const { return Pre{pix < n_pix ? __ldg(T + pix) : 1.0f}; }
    __device__ __forceinline__ void end(int64_t pix, const uint32_t (&r)[kRowAccStride], Pre pre, bool fail,
                                        unsigned char *) const
    {
        float best = -__int_as_float(0x7f800000);
        int arg = 0;
#pragma unroll
        for (int q = 0; q < static_cast<int>(kRowAccStride); ++q) {
            const float v = __uint_as_float(r[q]);
            if (q < n_q && v > best) {
                best = v;
                arg = q;
            }
        }
        if (logits && pix < n_pix) {
            __nv_bfloat16 *row = logits + pix * n_q;
            if ((n_q & 1) == 0) {
                // even row length: 4-byte aligned pairs, never past the row
#pragma unroll
                for (int q = 0; q < static_cast<int>(kRowAccStride); q += 2)
                    if (q < n_q)
                        *reinterpret_cast<__nv_bfloat162 *>(row + q) =
                            __floats2bfloat162_rn(__uint_as_float(r[q]), __uint_as_float(r[q + 1]));
            } else {
#pragma unroll
                for (int q = 0; q < static_cast<int>(kRowAccStride); ++q)
                    if (q < n_q) row[q] = __float2bfloat16_rn(__uint_as_float(r[q]));
            }
        }
        if (pix < n_pix && !fail) ids[pix] = (1.0f - pre.T < 1e-4f) ? -1 : arg;
    }
};

} // namespace

cudaError_t launch_decode(const void *F, int64_t n_pix, int D, const void *Q, int n_q, const float *T, int32_t *ids,
                          void *logits, DevStatus *status, cudaStream_t st, const char **why)
{
    const DecodeEpi epi{n_pix, n_q, T, ids, static_cast<__nv_bfloat16 *>(logits)};
    return launch_row_gemm(F, n_pix, D, Q, n_q, 0, epi, status, st, why);
}

} // namespace psi
