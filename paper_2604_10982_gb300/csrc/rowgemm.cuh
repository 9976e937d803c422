// A row-tile GEMM pipeline on the 5th-generation tensor cores, shared by the
// query decode and the instance-label kernels.
//
// Persistent CTAs walk 128-row tiles of A [rows x D] (BF16, K-major). TMA
// loads each [128 x D] tile (128-byte swizzle) into a shared-memory ring of
// Epi::kStages stages: 4 with one CTA per SM, or 2 with two CTAs per SM, which
// hides the latency of an epilogue that computes per row (the argmax of the
// decode, the softmax of the labels) behind the other CTA; one thread issues
// tcgen05.mma (M=128, N=n_pad, K=16 per instruction,
// FP32 accumulation in TMEM) against B [n_b x D] (BF16, resident in shared
// memory) into one of two TMEM accumulators, so the MMA of tile i+1 overlaps
// the epilogue of tile i. Each thread owns one row (TMEM lane): it reads the
// row's n_pad results with tcgen05.ld and hands them to the epilogue functor
// (prepare: per-CTA shared data; begin: loads issued before the TMEM read;
// end: the row's results). Every wait is bounded.
#pragma once

#include "tc.cuh"

namespace psi {
namespace tc {

constexpr int kRowM = 128;              // rows per tile (TMEM lanes)
constexpr int kRowThreads = 128;        // 4 warps: TMEM lane quarters 0..3
constexpr uint32_t kRowTmemCols = 256;
constexpr uint32_t kRowAccStride = 128; // column offset of the second accumulator

struct RowGemm {
    int64_t rows;
    int D;
    int n_pad;
    DevStatus *status;
};

// stages of the ring -> CTAs per SM (each CTA holds 256 TMEM columns: two fill TMEM)
__host__ __device__ constexpr int row_ctas_per_sm(int stages) { return stages <= 2 ? 2 : 1; }

template <class Epi>
__global__ void __launch_bounds__(kRowThreads, row_ctas_per_sm(Epi::kStages))
    row_gemm_kernel(const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_q, RowGemm p,
                    Epi epi)
{
    constexpr int kRowStages = Epi::kStages;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned carve-up: [stages][D/64 atoms][128 rows][128 B], then Q
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int atoms = p.D / 64;
    const uint32_t stage_bytes = static_cast<uint32_t>(atoms) * kRowM * 128;
    unsigned char *q_smem = base + kRowStages * stage_bytes;
    const uint32_t q_atom_bytes = static_cast<uint32_t>(p.n_pad) * 128;
    unsigned char *epi_smem = q_smem + atoms * q_atom_bytes; // the epilogue's own shared data
    __shared__ uint64_t full[kRowStages];
    __shared__ uint64_t mma_bar[2];
    __shared__ uint64_t q_bar;
    __shared__ uint32_t tmem_base_sh;

    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = (p.rows + kRowM - 1) / kRowM;
    const int my_n = blockIdx.x < n_tiles ? static_cast<int>((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const uint32_t tile_tx = stage_bytes;
    const uint32_t idesc = idesc_bf16(kRowM, p.n_pad);

    if (tid == 0) {
        for (int s = 0; s < kRowStages; ++s) mbar_init(&full[s], 1);
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        mbar_init(&q_bar, 1);
        fence_mbar_init();
    }
    epi.prepare(epi_smem, tid);
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kRowTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto tile_of = [&](int i) { return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(i) * gridDim.x; };
    auto issue_tile = [&](int i) {
        const int s = i % kRowStages;
        unsigned char *dst = base + s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], tile_tx);
        const int y = static_cast<int>(tile_of(i) * kRowM);
        for (int a = 0; a < atoms; ++a) tma_load_2d(dst + a * (kRowM * 128), &map_f, a * 64, y, &full[s]);
    };
    auto issue_mma = [&](int i) {
        const int s = i % kRowStages;
        const uint32_t a_base = smem_u32(base + s * stage_bytes);
        const uint32_t b_base = smem_u32(q_smem);
        const uint32_t d = tmem + (i & 1) * kRowAccStride;
        for (int k = 0; k < p.D / 16; ++k) {
            const int at = k >> 2, kin = k & 3;
            const uint64_t ad = sw128_desc(a_base + at * (kRowM * 128) + kin * 32);
            const uint64_t bd = sw128_desc(b_base + at * q_atom_bytes + kin * 32);
            mma_bf16(d, ad, bd, idesc, k > 0 ? 1u : 0u);
        }
        mma_commit(&mma_bar[i & 1]);
    };

    // thread 0 bookkeeping: loads issued / waited, MMA groups issued; all
    // threads wait on the MMA groups in order (m_waited).
    int t_issued = 0, t_waited = 0, m_issued = 0, m_waited = 0;
    bool q_pending = false;
    bool fail = false;
    if (tid == 0 && my_n > 0) {
        mbar_arrive_expect_tx(&q_bar, static_cast<uint32_t>(atoms) * q_atom_bytes);
        for (int a = 0; a < atoms; ++a) tma_load_2d(q_smem + a * q_atom_bytes, &map_q, a * 64, 0, &q_bar);
        q_pending = true;
        for (; t_issued < kRowStages && t_issued < my_n; ++t_issued) issue_tile(t_issued);
        fail = !mbar_wait(&q_bar, 0, p.status, kSiteDecodeQ);
        q_pending = fail;
        if (!fail) fail = !mbar_wait(&full[0], 0, p.status, kSiteDecodeLoad);
        if (!fail) {
            t_waited = 1;
            tc_fence_after();
            issue_mma(0);
            m_issued = 1;
        }
    }
    bool stop = __syncthreads_or(fail) != 0;

    for (int i = 0; i < my_n && !stop; ++i) {
        fail = false;
        if (tid == 0 && i + 1 < my_n) {
            if (mbar_wait(&full[(i + 1) % kRowStages], ((i + 1) / kRowStages) & 1, p.status, kSiteDecodeLoad)) {
                t_waited = i + 2;
                tc_fence_after();
                issue_mma(i + 1);
                m_issued = i + 2;
            } else {
                fail = true;
            }
        }
        if (mbar_wait(&mma_bar[i & 1], (i >> 1) & 1, p.status, kSiteDecodeMma))
            m_waited = i + 1;
        else
            fail = true;
        tc_fence_after();
        if (tid == 0 && !fail && i + kRowStages < my_n) {
            issue_tile(i + kRowStages);
            t_issued = i + kRowStages + 1;
        }
        // epilogue: one row (TMEM lane) per thread; all of the row's columns
        // are requested before a single wait
        const int64_t row = tile_of(i) * kRowM + wid * 32 + lane;
        const typename Epi::Pre pre = epi.begin(row);
        const uint32_t tacc = tmem + (i & 1) * kRowAccStride + (static_cast<uint32_t>(wid * 32) << 16);
        uint32_t r[kRowAccStride];
#pragma unroll
        for (int c0 = 0; c0 < static_cast<int>(kRowAccStride); c0 += 16)
            if (c0 < p.n_pad) tmem_ld16_async(tacc + c0, r + c0);
        tmem_wait_ld();
        epi.end(row, r, pre, fail, epi_smem);
        tc_fence_before();
        stop = __syncthreads_or(fail) != 0;
    }
    // after a give-up, let every started copy and MMA group land (bounded)
    // before TMEM and shared memory are released
    if (tid == 0) {
        if (q_pending) mbar_wait(&q_bar, 0, nullptr);
        for (int i = t_waited; i < t_issued; ++i) mbar_wait(&full[i % kRowStages], (i / kRowStages) & 1, nullptr);
        for (int i = m_waited; i < m_issued; ++i) mbar_wait(&mma_bar[i & 1], (i >> 1) & 1, nullptr);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRowTmemCols) : "memory");
    }
}


// rows x D times n_b x D, both BF16 row-major with 16-byte aligned rows;
// D in {64, 128}, 1 <= n_b <= 128. epi_smem_bytes: shared data of the epilogue.
template <class Epi>
cudaError_t launch_row_gemm(const void *A, int64_t rows, int D, const void *B, int n_b, size_t epi_smem_bytes,
                            const Epi &epi, DevStatus *status, cudaStream_t st, const char **why)
{
    constexpr int kRowStages = Epi::kStages;
    constexpr int ctas = row_ctas_per_sm(kRowStages);
    const int n_pad = ((n_b + 15) / 16) * 16;
    CUtensorMap map_a, map_b;
    if (!encode_2d_bf16(&map_a, A, static_cast<uint64_t>(D), static_cast<uint64_t>(rows), 64, kRowM) ||
        !encode_2d_bf16(&map_b, B, static_cast<uint64_t>(D), static_cast<uint64_t>(n_b), 64, static_cast<uint32_t>(n_pad))) {
        *why = "cuTensorMapEncodeTiled failed";
        return cudaErrorInvalidValue;
    }
    RowGemm p{rows, D, n_pad, status};
    // shared memory of at least 120 KB (one CTA per SM) or 80 KB (two): never
    // more CTAs on an SM than their 256 TMEM columns each can be granted at once
    const size_t smem = std::max<size_t>(ctas == 1 ? 120 * 1024 : 80 * 1024,
                                         1024 + static_cast<size_t>(kRowStages) * (D / 64) * kRowM * 128 +
                                             static_cast<size_t>(D / 64) * n_pad * 128 + epi_smem_bytes);
    if (ctas == 2 && 3 * smem <= 228 * 1024) {
        *why = "row GEMM shared memory too small to keep a third CTA off the SM";
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(row_gemm_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (rows + kRowM - 1) / kRowM;
    const int grid = static_cast<int>(std::min<int64_t>(tiles, std::max(ctas * sms, 1)));
    row_gemm_kernel<Epi><<<grid, kRowThreads, smem, st>>>(map_a, map_b, p, epi);
    return cudaGetLastError();
}

} // namespace tc
} // namespace psi
