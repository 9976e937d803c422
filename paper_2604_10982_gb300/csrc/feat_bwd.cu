// a5, feature part: the adjoint of the Top-K feature sum F = sum_{j in K}
// f_j omega_j (Sec. 5) from the forward's saved selection.
//
// For each pixel the forward keeps the selected surfels (ids, list order) and
// their weights omega_j. The feature terms of the adjoint then need no walk
// over the tile list:
//     kd_j     = <gF, f_j>                 (enters s_j of the list walk)
//     dL/df_j += omega_j gF                (summed over the pixels selecting j)
// One CTA per 16x16 tile, one thread per pixel (same pixel layout as the
// compositing kernels). kd is written per (pixel, slot) for the list walk.
// dL/df is aggregated per warp: the warp visits the distinct surfels its 32
// pixels selected (ascending id), accumulates omega gF over the selecting
// pixels with lanes across channels (coalesced gF rows), and adds the row to
// dL/df with one 16-byte atomic per lane.
#include "raster.cuh"

namespace psi {
namespace {

using namespace raster;

struct FeatBwdArgs {
    const void *feat;
    const float *fscale;
    int D;
    bool wide; // feature rows read 32 bytes at a time
    const int32_t *topk_ids; // [P_total, K]
    const float *topk_w;     // [P_total, K]
    const float *g_F;        // [P_total, D]
    float *kd;               // [P_total, K]
    float *g_feat;           // [N, D] or NULL
    DevStatus *status;
};

template <int KMAX, int DT>
__global__ void __launch_bounds__(256) feat_bwd_kernel(const __grid_constant__ FrameParams fp, FeatBwdArgs a)
{
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t tile = blockIdx.x;
    const int v = view_of_tile(fp, tile);
    const ViewParams &cam = fp.v[v];
    const int local = static_cast<int>(tile - cam.tile_base);
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
    int lxi, lyi;
    pixel_of_thread(tid, lxi, lyi);
    const int px = tx * kTile + lxi, py = ty * fp.tile_h + lyi; // blockDim = 16 x tile height
    const bool inside = px < cam.W && py < cam.H;
    const int64_t pix = cam.pix_base + static_cast<int64_t>(min(py, cam.H - 1)) * cam.W + min(px, cam.W - 1);
    const int K = fp.top_k;

    int id[KMAX];
    float w[KMAX];
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        id[s] = (inside && s < K) ? a.topk_ids[pix * K + s] : -1;
        // debug builds: a saved id must be -1 or a surfel of the table
        if (!PSI_CHECK(id[s] >= -1 && id[s] < fp.n, kChkFeatRow, a.status)) id[s] = -1;
        w[s] = id[s] >= 0 ? a.topk_w[pix * K + s] : 0.0f;
    }

    // kd_j = <gF, f_j> (dequantised f: per-channel scale folded into gF)
    if (inside) {
        float kd[KMAX];
#pragma unroll
        for (int s = 0; s < KMAX; ++s) kd[s] = 0.0f;
        for (int c0 = 0; c0 < a.D; c0 += 16) {
            float g[16];
#pragma unroll
            for (int c = 0; c < 16; c += 4) {
                const float4 q = __ldg(reinterpret_cast<const float4 *>(a.g_F + pix * a.D + c0 + c));
                const float sc0 = a.fscale ? __ldg(a.fscale + c0 + c) : 1.0f;
                const float sc1 = a.fscale ? __ldg(a.fscale + c0 + c + 1) : 1.0f;
                const float sc2 = a.fscale ? __ldg(a.fscale + c0 + c + 2) : 1.0f;
                const float sc3 = a.fscale ? __ldg(a.fscale + c0 + c + 3) : 1.0f;
                g[c] = q.x * sc0;
                g[c + 1] = q.y * sc1;
                g[c + 2] = q.z * sc2;
                g[c + 3] = q.w * sc3;
            }
#pragma unroll
            for (int s = 0; s < KMAX; ++s) {
                if (id[s] < 0) continue;
                float f[16];
                load_feat<DT, 16>(a.feat, id[s], a.D, c0, f, a.wide);
                float acc = kd[s];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc = __fmaf_rn(g[c], f[c], acc);
                kd[s] = acc;
            }
        }
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s < K) a.kd[pix * K + s] = kd[s];
    }
    if (!a.g_feat) return;

    // dL/df_j += omega_j gF, one distinct surfel of the warp at a time
    const int nv = a.D >> 2; // float4 chunks per row (D <= 256: lanes cover lane and lane + 32)
    uint32_t used = 0;       // slots already added
    while (true) {
        uint32_t mine = 0xffffffffu;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (id[s] >= 0 && !((used >> s) & 1u)) mine = min(mine, static_cast<uint32_t>(id[s]));
        const uint32_t cur = __reduce_min_sync(0xffffffffu, mine);
        if (cur == 0xffffffffu) break;
        float wsel = 0.0f;
        bool has = false;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (static_cast<uint32_t>(id[s]) == cur) { // ids are distinct within a pixel's set
                wsel = w[s];
                has = true;
                used |= 1u << s;
            }
        uint32_t m = __ballot_sync(0xffffffffu, has);
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        while (m) {
            // up to four selecting pixels per round so their gF loads overlap
            int Ls[4];
            int nL = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                Ls[q] = m ? __ffs(m) - 1 : 0;
                if (m) {
                    m &= m - 1;
                    ++nL;
                }
            }
            float wq[4];
            float4 g0[4], g1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool on = q < nL;
                wq[q] = __shfl_sync(0xffffffffu, wsel, Ls[q]);
                const long long pL = __shfl_sync(0xffffffffu, static_cast<long long>(pix), Ls[q]);
                const float4 *row = reinterpret_cast<const float4 *>(a.g_F + pL * a.D);
                g0[q] = (on && lane < nv) ? __ldg(row + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                g1[q] = (on && lane + 32 < nv) ? __ldg(row + lane + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (!on) wq[q] = 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc0.x = fmaf(wq[q], g0[q].x, acc0.x);
                acc0.y = fmaf(wq[q], g0[q].y, acc0.y);
                acc0.z = fmaf(wq[q], g0[q].z, acc0.z);
                acc0.w = fmaf(wq[q], g0[q].w, acc0.w);
                acc1.x = fmaf(wq[q], g1[q].x, acc1.x);
                acc1.y = fmaf(wq[q], g1[q].y, acc1.y);
                acc1.z = fmaf(wq[q], g1[q].z, acc1.z);
                acc1.w = fmaf(wq[q], g1[q].w, acc1.w);
            }
        }
        float4 *dst = reinterpret_cast<float4 *>(a.g_feat + static_cast<int64_t>(cur) * a.D);
        if (lane < nv) atomicAdd(dst + lane, acc0);
        if (lane + 32 < nv) atomicAdd(dst + lane + 32, acc1);
    }
}

template <int KMAX>
cudaError_t launch_k(const FrameParams &fp, const FeatView &f, const FeatBwdArgs &a, cudaStream_t st)
{
    const unsigned grid = static_cast<unsigned>(fp.n_tiles_total);
    switch (f.dtype) {
    case PSI_BF16: feat_bwd_kernel<KMAX, PSI_BF16><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
    case PSI_FP8_E4M3: feat_bwd_kernel<KMAX, PSI_FP8_E4M3><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
    default: feat_bwd_kernel<KMAX, PSI_F32><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
    }
    return cudaGetLastError();
}

} // namespace

cudaError_t launch_feat_bwd(const FrameParams &fp, const FeatView &f, const int32_t *topk_ids, const float *topk_w,
                            const float *g_F, float *kd, float *g_feat, DevStatus *status, cudaStream_t st)
{
    if (fp.n_tiles_total == 0 || fp.top_k <= 0 || !f.data || !g_F) return cudaSuccess;
    FeatBwdArgs a{};
    a.feat = f.data;
    a.wide = feat_rows_wide(f.data, f.dim, f.dtype);
    a.fscale = f.scale;
    a.D = f.dim;
    a.topk_ids = topk_ids;
    a.topk_w = topk_w;
    a.g_F = g_F;
    a.kd = kd;
    a.g_feat = g_feat;
    a.status = status;
    if (fp.top_k <= 8) return launch_k<8>(fp, f, a, st);
    if (fp.top_k <= 16) return launch_k<16>(fp, f, a, st);
    return launch_k<32>(fp, f, a, st);
}

} // namespace psi
