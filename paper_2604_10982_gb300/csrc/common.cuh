// Internal declarations shared by the libpsi translation units (sm_103a only).
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "psi.h" // include/ is on the include path

namespace psi {

// Device status word layout (see psi_status_fetch): [0] OR of error codes as
// bits (1 << code), [1] code of the first bounded wait that gave up,
// [2..3] int64 pairs required on overflow (these 16 bytes are read and
// cleared by psi_status_fetch); then the context's wait limit in ns
// (psi_ctx_set_wait_limit_ns), kept across fetches.
struct DevStatus {
    int32_t flags;
    int32_t wait_site;
    unsigned long long required_pairs;
    unsigned long long wait_limit_ns;
    unsigned int work[4]; // persistent compositing: tile counter and finished-CTA count (forward, adjoint)
};
constexpr size_t kDevStatusReportBytes = 16;

__device__ __forceinline__ void raise_status(DevStatus *st, int code)
{
    if (st) atomicOr(&st->flags, 1 << code);
}

// Bounds checks of the debug build (PSI_DEBUG): indices that come from data
// are checked before use; a failure records 100 + the site in the status
// word's site field, raises PSI_ERR_BOUNDS and the caller clamps the access.
// The release build compiles the checks away.
enum CheckSite { kChkTile = 1, kChkRange = 2, kChkRecord = 3, kChkFeatRow = 4, kChkLast = 5 };
#ifdef PSI_DEBUG
__device__ __forceinline__ bool check_index(bool ok, int site, DevStatus *st)
{
    if (!ok && st) {
        atomicCAS(&st->wait_site, 0, 100 + site);
        raise_status(st, PSI_ERR_BOUNDS);
    }
    return ok;
}
#define PSI_CHECK(cond, site, st) ::psi::check_index((cond), (site), (st))
#else
#define PSI_CHECK(cond, site, st) true
#endif

// wait sites (reported by psi_status_fetch on PSI_ERR_TIMEOUT)
enum WaitSite {
    kSiteRenderFwd = 1,
    kSiteRenderBwdA = 2,
    kSiteRenderBwdB = 3,
    kSiteDecodeQ = 4,
    kSiteDecodeLoad = 5,
    kSiteDecodeMma = 6,
    kSiteDrain = 7,
    kSiteSort = 8
};

struct ViewParams {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    uint32_t tile_base;
    int32_t pad;
    int64_t pix_base;
};

struct FrameParams {
    int32_t n_views;
    int32_t mode;
    int64_t n;          // surfels
    int32_t tile_w, tile_h;
    float chi2, z_near, t_eps;
    int32_t opacity_radius;
    int32_t top_k;
    int32_t lowpass; // 2DGS object-space low-pass filter
    uint32_t n_tiles_total;
    int64_t n_pix_total;
    ViewParams v[PSI_MAX_VIEWS];
};

// view that owns global tile t (views are few: linear scan)
__device__ __forceinline__ int view_of_tile(const FrameParams &fp, uint32_t t)
{
    int v = 0;
    for (int k = 1; k < fp.n_views; ++k)
        if (t >= fp.v[k].tile_base) v = k;
    return v;
}

// ---------------------------------------------------------------- waits
// Every spin in this library is bounded by wall time read from %globaltimer:
// by the context's limit (1 s unless psi_ctx_set_wait_limit_ns changed it) for
// the waits of the pipelines, and always by the fixed 1 s for the drains that
// let in-flight copies and MMA groups land after a give-up, so that a short
// limit can never release shared memory or TMEM that a copy still writes.
constexpr unsigned long long kWaitLimitNs = 1000000000ull; // 1 s

__device__ __forceinline__ unsigned long long wait_limit(const DevStatus *st)
{
    if (!st) return kWaitLimitNs;
    const unsigned long long l = *reinterpret_cast<const volatile unsigned long long *>(&st->wait_limit_ns);
    return l ? l : kWaitLimitNs;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; returns false (and raises TIMEOUT with
// the wait site) on give-up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, DevStatus *st, int site = 0)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long limit = site == kSiteDrain ? kWaitLimitNs : wait_limit(st);
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit) {
            if (st) {
                atomicCAS(&st->wait_site, 0, site);
                raise_status(st, PSI_ERR_TIMEOUT);
            }
            return false;
        }
    }
    return true;
}

// 1D bulk copy global -> shared through the TMA engine, completion counted on bar.
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gsrc, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- launchers
// (host side; defined in the kernel translation units)
void fill_frame_params(FrameParams &fp, const psi_camera *cams, int n_views, const psi_render_opts *o, int64_t n);

cudaError_t launch_project(const FrameParams &fp, const psi_surfels &s, float4 *records, float4 *bin_records,
                           uint32_t *tiles_touched, cudaStream_t st);

size_t intersect_workspace_bytes(int64_t n_records);
cudaError_t launch_intersect(const FrameParams &fp, const float4 *bin_records, const uint32_t *tiles_touched,
                             uint64_t *keys, uint32_t *vals, int64_t capacity, int64_t *d_num_pairs, void *ws,
                             DevStatus *status, cudaStream_t st);

size_t sort_workspace_bytes(int64_t capacity);
cudaError_t launch_sort(uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs, int64_t capacity, int begin_bit,
                        int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total, void *ws, DevStatus *status,
                        cudaStream_t st);

constexpr int PSI_MAX_DEVICES_NOALLOC = PSI_SORT_NOALLOC_MAX_DEVICES;
cudaError_t launch_sort_noalloc(uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs, int64_t capacity,
                                int begin_bit, int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total,
                                DevStatus *status, cudaStream_t st, const char **why);

struct FeatView {
    const void *data;
    const float *scale;
    int dtype;
    int dim;
};

// Launch shapes of the compositing kernels (a4, a5), picked per workload by
// the autotuner: bit 0 builds the kernel for the alternative number of CTAs
// per SM (registers per thread against occupancy), bit 1 composites dense
// features (K = 0) 16 channels per pass instead of 32, bit 2 launches the
// persistent form (a few CTAs per SM fetching tiles from a counter), bit 3
// runs the adjoint's walk from saved state with a Top-K selection two pixels
// per lane instead of one. Every shape computes the same result.
constexpr int kShapeAltOcc = 1;
constexpr int kShapeAltChunk = 2;
constexpr int kShapePersistent = 4;
constexpr int kShapePairWalk = 8;
constexpr int kShapes = 16;
// channels per pass of the dense feature path for this shape
inline int render_channel_chunk(int D, int K, int shape)
{
    const int ch = (D % 32 == 0) ? 32 : 16;
    return (K == 0 && (shape & kShapeAltChunk)) ? 16 : ch;
}
// shapes that differ from shape 0 in something that exists for (D, K) and
// the kernel (pair_walk: the adjoint from saved state with K > 0)
inline bool render_shape_valid(int D, int K, int shape, bool pair_walk)
{
    if (shape < 0 || shape >= kShapes) return false;
    if ((shape & kShapePairWalk) && !pair_walk) return false;
    return !(shape & kShapeAltChunk) || (K == 0 && D % 32 == 0);
}

cudaError_t launch_render_fwd(const FrameParams &fp, const FeatView &f, const float4 *records, const uint32_t *vals,
                              const uint32_t *ranges, const psi_fwd_out &out, DevStatus *status, cudaStream_t st,
                              int shape);

size_t render_bwd_workspace_bytes(int64_t n_records, int64_t n_pix, int top_k);
cudaError_t launch_feat_bwd(const FrameParams &fp, const FeatView &f, const int32_t *topk_ids, const float *topk_w,
                            const float *g_F, float *kd, float *g_feat, DevStatus *status, cudaStream_t st);
cudaError_t launch_render_bwd(const FrameParams &fp, const psi_surfels &s, const FeatView &f, const float4 *records,
                              const uint32_t *vals, const uint32_t *ranges, const float *g_rgb, const float *g_F,
                              const float *g_T, const psi_fwd_out *saved, const psi_grads &g, void *ws,
                              DevStatus *status, cudaStream_t st, cudaEvent_t const (*time_ev)[2], int shape);

size_t attention_workspace_bytes(int64_t n, int C, int d, int n_q);
cudaError_t launch_attention(const psi_surfels &s, const void *feat, int C, const psi_camera &cam, float z_near,
                             const float *Q, int n_q, const float *WQ, const float *WK, const float *WV, int d,
                             float *out, void *ws, DevStatus *status, cudaStream_t st, const char **why);
cudaError_t launch_attention_bwd(const psi_surfels &s, const void *feat, int C, const float *Q, int n_q,
                                 const float *WQ, const float *WK, const float *WV, int d, const float *G_out,
                                 float *gQ, float *gWQ, float *gWK, float *gWV, float *g_feat, float *g_mu, void *ws,
                                 DevStatus *status, cudaStream_t st, const char **why);
cudaError_t launch_quantize(const float *f, int64_t n, int dim, int dtype, void *q, float *scale, cudaStream_t st);
// fill.cu: zero up to kFillMaxParts float buffers (NULL or empty ones skipped)
// with one small kernel (one CTA per SM)
constexpr int kFillMaxParts = 8;
cudaError_t launch_zero_parts(float *const *ptrs, const int64_t *counts, int n_parts, cudaStream_t st);
cudaError_t launch_frames(const float *q, int64_t n, float *tu, float *tv, cudaStream_t st);
cudaError_t launch_frames_bwd(const float *q, int64_t n, const float *g_tu, const float *g_tv, float *g_q,
                              cudaStream_t st);
cudaError_t launch_regularisers(const psi_surfels &s, const int32_t *node_of, const float *node_mu, const float *node_n,
                                int64_t n_nodes, float lambda_n, float w_geo, float w_iso, double *losses,
                                const psi_grads &g, DevStatus *status, cudaStream_t st);
cudaError_t launch_logits(const void *F, int64_t n, int D, const void *Q, int n_q, void *table, int ld, int out_bf16,
                          DevStatus *status, cudaStream_t st, const char **why);
cudaError_t launch_labels(const void *F, int64_t n, int D, const float *centres, const void *Q, int n_q,
                          const float *q_mu, const float *q_cov, void *labels, int ld, int out_bf16, DevStatus *status,
                          cudaStream_t st, const char **why);
cudaError_t launch_decode(const void *F, int64_t n_pix, int D, const void *Q, int n_q, const float *T, int32_t *ids,
                          void *logits, DevStatus *status, cudaStream_t st, const char **why);

// Exclusive scan of uint32 counts into uint64 offsets (reduce-then-scan,
// spin-free). Writes the total to *d_total (uint64). ws: scan_workspace_bytes(n).
size_t scan_workspace_bytes(int64_t n);
cudaError_t launch_scan_u32(const uint32_t *in, unsigned long long *out, int64_t n, unsigned long long *d_total,
                            void *ws, cudaStream_t st);

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

} // namespace psi
