// a6: query decode on the 5th-generation tensor cores.
//
// logits[p, q] = sum_c F[p, c] Q[q, c] (the feature similarity f_q^T f_g of
// Sec. 4.1, Eq. 4, before its monotone sigmoid), then the per-pixel argmax
// (lowest q on ties) as the panoptic id, -1 where nothing was rendered.
//
// Persistent CTAs walk 128-pixel tiles. TMA loads each [128 x D] BF16 tile
// (128-byte swizzle, K-major) into a 4-deep shared-memory ring; one thread
// issues tcgen05.mma (M=128, N=round16(Q), K=16 per instruction, FP32
// accumulation in TMEM) into one of two TMEM accumulators, so the MMA of tile
// i+1 overlaps the epilogue of tile i. Each epilogue warp reads its 32 TMEM
// lanes (one pixel per thread) with tcgen05.ld and reduces the row in
// registers. The query matrix stays resident in shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace psi {
namespace {

constexpr int kM = 128;          // pixels per tile (TMEM lanes)
constexpr int kStages = 4;
constexpr int kThreads = 128;    // 4 warps: TMEM lane quarters 0..3
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kAccStride = 128; // column offset of the second accumulator

struct DecodeParams {
    int64_t n_pix;
    int D;
    int n_q;
    int n_pad;
    const float *T;
    int32_t *ids;
    __nv_bfloat16 *logits;
    DevStatus *status;
};

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand in the canonical
// 128-byte swizzle layout -- 8-row groups of 128-byte rows, 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);       // start address
    d |= static_cast<uint64_t>(1) << 16;                       // leading byte offset (unused for swizzled K-major)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;               // stride byte offset: next 8-row group
    d |= static_cast<uint64_t>(1) << 46;                       // descriptor version (sm_100 family)
    d |= static_cast<uint64_t>(2) << 61;                       // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: D=F32, A=B=BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane; the values are valid
// only after tmem_wait_ld (several loads can be in flight before one wait).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t *r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1) decode_kernel(const __grid_constant__ CUtensorMap map_f,
                                                            const __grid_constant__ CUtensorMap map_q,
                                                            DecodeParams p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned carve-up: [stages][D/64 atoms][128 rows][128 B], then Q
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int atoms = p.D / 64;
    const uint32_t stage_bytes = static_cast<uint32_t>(atoms) * kM * 128;
    unsigned char *q_smem = base + kStages * stage_bytes;
    const uint32_t q_atom_bytes = static_cast<uint32_t>(p.n_pad) * 128;
    __shared__ uint64_t full[kStages];
    __shared__ uint64_t mma_bar[2];
    __shared__ uint64_t q_bar;
    __shared__ uint32_t tmem_base_sh;

    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int64_t n_tiles = (p.n_pix + kM - 1) / kM;
    const int my_n = blockIdx.x < n_tiles ? static_cast<int>((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const uint32_t tile_tx = stage_bytes;
    const uint32_t idesc = idesc_bf16(kM, p.n_pad);

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        mbar_init(&q_bar, 1);
        fence_mbar_init();
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    auto tile_of = [&](int i) { return static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(i) * gridDim.x; };
    auto issue_tile = [&](int i) {
        const int s = i % kStages;
        unsigned char *dst = base + s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], tile_tx);
        const int y = static_cast<int>(tile_of(i) * kM);
        for (int a = 0; a < atoms; ++a) tma_load_2d(dst + a * (kM * 128), &map_f, a * 64, y, &full[s]);
    };
    auto issue_mma = [&](int i) {
        const int s = i % kStages;
        const uint32_t a_base = smem_u32(base + s * stage_bytes);
        const uint32_t b_base = smem_u32(q_smem);
        const uint32_t d = tmem + (i & 1) * kAccStride;
        for (int k = 0; k < p.D / 16; ++k) {
            const int at = k >> 2, kin = k & 3;
            const uint64_t ad = sw128_desc(a_base + at * (kM * 128) + kin * 32);
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
        for (; t_issued < kStages && t_issued < my_n; ++t_issued) issue_tile(t_issued);
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
            if (mbar_wait(&full[(i + 1) % kStages], ((i + 1) / kStages) & 1, p.status, kSiteDecodeLoad)) {
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
        if (tid == 0 && !fail && i + kStages < my_n) {
            issue_tile(i + kStages);
            t_issued = i + kStages + 1;
        }
        // epilogue: one pixel (TMEM lane) per thread; all of the row's
        // columns are requested before a single wait
        const int64_t pix = tile_of(i) * kM + wid * 32 + lane;
        const float Tp = pix < p.n_pix ? __ldg(p.T + pix) : 1.0f;
        const uint32_t tacc = tmem + (i & 1) * kAccStride + (static_cast<uint32_t>(wid * 32) << 16);
        uint32_t r[kAccStride];
#pragma unroll
        for (int c0 = 0; c0 < static_cast<int>(kAccStride); c0 += 16)
            if (c0 < p.n_pad) tmem_ld16_async(tacc + c0, r + c0);
        tmem_wait_ld();
        float best = -__int_as_float(0x7f800000);
        int arg = 0;
#pragma unroll
        for (int q = 0; q < static_cast<int>(kAccStride); ++q) {
            const float v = __uint_as_float(r[q]);
            if (q < p.n_q && v > best) {
                best = v;
                arg = q;
            }
        }
        if (p.logits && pix < p.n_pix) {
            __nv_bfloat16 *row = p.logits + pix * p.n_q;
            if ((p.n_q & 1) == 0) {
                // even row length: 4-byte aligned pairs, never past the row
#pragma unroll
                for (int q = 0; q < static_cast<int>(kAccStride); q += 2)
                    if (q < p.n_q)
                        *reinterpret_cast<__nv_bfloat162 *>(row + q) =
                            __floats2bfloat162_rn(__uint_as_float(r[q]), __uint_as_float(r[q + 1]));
            } else {
#pragma unroll
                for (int q = 0; q < static_cast<int>(kAccStride); ++q)
                    if (q < p.n_q) row[q] = __float2bfloat16_rn(__uint_as_float(r[q]));
            }
        }
        if (pix < p.n_pix && !fail) p.ids[pix] = (1.0f - Tp < 1e-4f) ? -1 : arg;
        tc_fence_before();
        stop = __syncthreads_or(fail) != 0;
    }
    // after a give-up, let every started copy and MMA group land (bounded)
    // before TMEM and shared memory are released
    if (tid == 0) {
        if (q_pending) mbar_wait(&q_bar, 0, nullptr);
        for (int i = t_waited; i < t_issued; ++i) mbar_wait(&full[i % kStages], (i / kStages) & 1, nullptr);
        for (int i = m_waited; i < m_issued; ++i) mbar_wait(&mma_bar[i & 1], (i >> 1) & 1, nullptr);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool encode_2d_bf16(CUtensorMap *map, const void *ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
                    uint32_t box_outer)
{
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

} // namespace

cudaError_t launch_decode(const void *F, int64_t n_pix, int D, const void *Q, int n_q, const float *T, int32_t *ids,
                          void *logits, DevStatus *status, cudaStream_t st, const char **why)
{
    const int n_pad = ((n_q + 15) / 16) * 16;
    CUtensorMap map_f, map_q;
    if (!encode_2d_bf16(&map_f, F, static_cast<uint64_t>(D), static_cast<uint64_t>(n_pix), 64, kM) ||
        !encode_2d_bf16(&map_q, Q, static_cast<uint64_t>(D), static_cast<uint64_t>(n_q), 64, static_cast<uint32_t>(n_pad))) {
        *why = "cuTensorMapEncodeTiled failed";
        return cudaErrorInvalidValue;
    }
    DecodeParams p{n_pix, D, n_q, n_pad, T, ids, static_cast<__nv_bfloat16 *>(logits), status};
    // at least 120 KB so one CTA owns each SM (its 256 TMEM columns never wait on a co-resident CTA)
    const size_t smem = std::max<size_t>(120 * 1024, 1024 + static_cast<size_t>(kStages) * (D / 64) * kM * 128 +
                                                         static_cast<size_t>(D / 64) * n_pad * 128);
    cudaError_t e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (n_pix + kM - 1) / kM;
    const int grid = static_cast<int>(std::min<int64_t>(tiles, std::max(sms, 1)));
    decode_kernel<<<grid, kThreads, smem, st>>>(map_f, map_q, p);
    return cudaGetLastError();
}

} // namespace psi
