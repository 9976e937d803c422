// a5, feature part: the adjoint of the Top-K feature sum F = sum_{j in K}
// f_j omega_j (Sec. 5) from the forward's saved selection.
//
// For each pixel the forward keeps the selected surfels (ids, list order) and
// their weights omega_j. The feature terms of the adjoint then need no walk
// over the tile list:
//     kd_j     = <gF, f_j>                 (enters s_j of the list walk)
//     dL/df_j += omega_j gF                (summed over the pixels selecting j)
// One CTA per tile, one thread per pixel (same pixel layout as the
// compositing kernels). kd is written per (pixel, slot) for the list walk.
// dL/df is aggregated per tile in shared memory (see the kernel), so that each
// pixel's gF row is read once per 32-channel chunk rather than once per
// selected surfel.
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

// the shared accumulator of the dL/df pass: rows, the id table (power of two)
constexpr int kAccRows = 128;
constexpr int kHashBits = 11;
constexpr int kHash = 1 << kHashBits;
constexpr uint8_t kRowDirect = 0xFE; // past the accumulator: added to dL/df directly
constexpr uint8_t kRowNone = 0xFF;   // empty slot

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
    if (!a.g_feat) return; // uniform over the CTA

    // dL/df_j += omega_j gF. The tile's distinct selected surfels get rows of
    // a shared accumulator (ids hashed into a shared table, rows handed out
    // in table order); per chunk of 32 channels each warp walks its 32 pixels
    // with lanes across channels -- one coalesced read of each gF row chunk --
    // and adds omega gF to the row of every surfel the pixel selected (shared
    // atomics, conflict-free: lane = channel); the rows then go to dL/df with
    // one coalesced atomic pass each. Surfels past the accumulator's rows (or
    // a full table) are added to dL/df directly.
    __shared__ int s_key[kHash];
    __shared__ int s_row[kHash];
    __shared__ int s_id[kAccRows];
    __shared__ unsigned int s_n;
    __shared__ float s_acc[kAccRows][32];
    __shared__ uint8_t s_d[256][KMAX];
    const int nthr = blockDim.x, wid = tid >> 5, nwarp = nthr >> 5;
    for (int h = tid; h < kHash; h += nthr) s_key[h] = -1;
    if (tid == 0) s_n = 0;
    __syncthreads();
    auto home = [](int id) { return static_cast<int>((static_cast<uint32_t>(id) * 2654435761u) >> (32 - kHashBits)); };
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        if (id[s] < 0) continue;
        int h = home(id[s]);
        for (int probe = 0; probe < kHash; ++probe, h = (h + 1) & (kHash - 1)) {
            const int prev = atomicCAS(&s_key[h], -1, id[s]);
            if (prev == -1 || prev == id[s]) break;
        }
    }
    __syncthreads();
    for (int h = tid; h < kHash; h += nthr) {
        const int k = s_key[h];
        if (k >= 0) {
            const unsigned int r = atomicAdd(&s_n, 1u);
            s_row[h] = r < kAccRows ? static_cast<int>(r) : kRowDirect;
            if (r < kAccRows) s_id[r] = k;
        }
    }
    __syncthreads();
    const int nrows = min(static_cast<int>(s_n), kAccRows);
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        uint8_t d = kRowNone;
        if (id[s] >= 0) {
            d = kRowDirect; // unless found below
            int h = home(id[s]);
            for (int probe = 0; probe < kHash; ++probe, h = (h + 1) & (kHash - 1)) {
                const int k = s_key[h];
                if (k == id[s]) {
                    d = static_cast<uint8_t>(s_row[h]);
                    break;
                }
                if (k == -1) break;
            }
        }
        s_d[tid][s] = d;
    }
    __syncthreads();
    for (int c0 = 0; c0 < a.D; c0 += 32) {
        for (int k = tid; k < nrows * 32; k += nthr) (&s_acc[0][0])[k] = 0.0f;
        __syncthreads();
        const int c = c0 + lane;
        const bool on = c < a.D;
#pragma unroll 1
        for (int q = 0; q < 32; ++q) {
            const long long pq = __shfl_sync(0xffffffffu, static_cast<long long>(pix), q);
            if (!__shfl_sync(0xffffffffu, inside, q)) continue;
            const float g = on ? __ldg(a.g_F + pq * a.D + c) : 0.0f;
#pragma unroll
            for (int s = 0; s < KMAX; ++s) {
                const uint8_t d = s_d[wid * 32 + q][s];
                const float wq = __shfl_sync(0xffffffffu, w[s], q);
                const int iq = __shfl_sync(0xffffffffu, id[s], q);
                if (d == kRowNone || !on) continue;
                if (d < kAccRows)
                    atomicAdd(&s_acc[d][lane], wq * g);
                else
                    atomicAdd(a.g_feat + static_cast<int64_t>(iq) * a.D + c, wq * g);
            }
        }
        __syncthreads();
        for (int r = wid; r < nrows; r += nwarp)
            if (on) atomicAdd(a.g_feat + static_cast<int64_t>(s_id[r]) * a.D + c, s_acc[r][lane]);
        __syncthreads();
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
