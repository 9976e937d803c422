// a5, feature part: the adjoint of the Top-K feature sum F = sum_{j in K}
// f_j omega_j (Sec. 5) from the forward's saved selection.
//
// For each pixel the forward keeps the selected surfels (ids, list order) and
// their weights omega_j. The feature terms of the adjoint then need no walk
// over the tile list:
//     kd_j     = <gF, f_j>                 (enters s_j of the list walk)
//     dL/df_j += omega_j gF                (summed over the pixels selecting j)
// One CTA per 16x16 tile (16 x TH for other tile heights), one thread per
// pixel (same pixel layout as the compositing kernels) for the bookkeeping;
// the arithmetic runs with lanes across channels. Each warp visits the
// distinct surfels its 32 pixels selected, in ascending id (every lane keeps
// its set sorted by id, so its next surfel is always its first slot). For one
// surfel the warp reads the feature row once and the gF row of each selecting
// pixel once (both coalesced): the row feeds omega gF into the surfel's
// dL/df (one 16-byte atomic per lane per surfel) and, through a cross-lane
// sum, the pixel's kd.
#include "raster.cuh"

namespace psi {
namespace {

using namespace raster;

struct FeatBwdArgs {
    const void *feat;
    const float *fscale;
    int D;
    const int32_t *topk_ids; // [P_total, K]
    const float *topk_w;     // [P_total, K]
    const float *g_F;        // [P_total, D]
    float *kd;               // [P_total, K]
    float *g_feat;           // [N, D] or NULL
    DevStatus *status;
};

// Sum 4 per-lane values over the warp (a transposing butterfly, 6 shuffles):
// afterwards lane l holds the total of value index l >> 3.
__device__ __forceinline__ float warp_transpose_sum4(float v[4], int lane)
{
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool hi = lane & 16;
        const float send = hi ? v[k] : v[k + 2];
        const float keep = hi ? v[k + 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    {
        const bool hi = lane & 8;
        const float send = hi ? v[0] : v[1];
        const float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 4);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// Slot indices of a pixel's sorted set: KMAX <= 8 packs them as nibbles of
// one word (fewer registers: four CTAs per SM fit), larger sets keep an array.
template <int KMAX, bool PACK = (KMAX <= 8)>
struct SlotOrder {
    int so[KMAX];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int s = 0; s < KMAX; ++s) so[s] = s;
    }
    __device__ __forceinline__ void swap(int s)
    {
        const int t = so[s];
        so[s] = so[s + 1];
        so[s + 1] = t;
    }
    __device__ __forceinline__ int first() const { return so[0]; }
    __device__ __forceinline__ void pop()
    {
#pragma unroll
        for (int s = 0; s + 1 < KMAX; ++s) so[s] = so[s + 1];
    }
};
template <int KMAX>
struct SlotOrder<KMAX, true> {
    uint32_t so; // nibble s: the saved slot of sorted position s
    __device__ __forceinline__ void init() { so = 0x76543210u; }
    __device__ __forceinline__ void swap(int s)
    {
        const uint32_t x = ((so >> (4 * s)) ^ (so >> (4 * s + 4))) & 0xFu;
        so ^= (x << (4 * s)) | (x << (4 * s + 4));
    }
    __device__ __forceinline__ int first() const { return static_cast<int>(so & 0xFu); }
    __device__ __forceinline__ void pop() { so >>= 4; }
};

// The pixel's saved set sorted by surfel id (odd-even transposition
// network; empty slots hold 0xffffffff and sort last), with each slot's
// weight and its index in the saved set.
template <int KMAX>
__device__ __forceinline__ void load_sorted_set(const FrameParams &fp, const FeatBwdArgs &a, bool inside, int64_t pix,
                                                uint32_t id[KMAX], float w[KMAX], SlotOrder<KMAX> &so)
{
    const int K = fp.top_k;
    so.init();
#pragma unroll
    for (int s = 0; s < KMAX; ++s) {
        int i = (inside && s < K) ? a.topk_ids[pix * K + s] : -1;
        // debug builds: a saved id must be -1 or a surfel of the table
        if (!PSI_CHECK(i >= -1 && i < fp.n, kChkFeatRow, a.status)) i = -1;
        id[s] = static_cast<uint32_t>(i);
        w[s] = i >= 0 ? a.topk_w[pix * K + s] : 0.0f;
    }
#pragma unroll
    for (int round = 0; round < KMAX; ++round) {
#pragma unroll
        for (int s = (round & 1); s + 1 < KMAX; s += 2) {
            if (id[s] > id[s + 1]) {
                const uint32_t ti = id[s];
                id[s] = id[s + 1];
                id[s + 1] = ti;
                const float tw = w[s];
                w[s] = w[s + 1];
                w[s + 1] = tw;
                so.swap(s);
            }
        }
    }
}

// NCH: 16-byte channel chunks per lane (1: D <= 128, 2: D <= 256).
template <int KMAX, int DT, int NCH>
__global__ void __launch_bounds__(256, (KMAX <= 8 && NCH == 1) ? 4 : 1) feat_bwd_kernel(const __grid_constant__ FrameParams fp, FeatBwdArgs a)
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

    // the pixel's selected set sorted by surfel id (empty slots: 0xffffffff,
    // last), with each slot's weight and its index in the saved set
    uint32_t id[KMAX];
    float w[KMAX];
    SlotOrder<KMAX> so;
    load_sorted_set<KMAX>(fp, a, inside, pix, id, w, so);

    // lane l owns channels [4l, 4l + 4) and [4l + 128, 4l + 132) (D <= 256)
    const int nv = a.D >> 2;
    const bool c0on = lane < nv, c1on = NCH > 1 && lane + 32 < nv;
    float4 sc0 = make_float4(1.f, 1.f, 1.f, 1.f), sc1 = sc0;
    if (a.fscale) {
        const float *p = a.fscale + 4 * lane; // the scale array has no alignment beyond 4 bytes
        if (c0on) sc0 = make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
        if (c1on) sc1 = make_float4(__ldg(p + 128), __ldg(p + 129), __ldg(p + 130), __ldg(p + 131));
    }
    const unsigned lt = (1u << lane) - 1u; // lanes below this one
    while (true) {
        const uint32_t cur = __reduce_min_sync(0xffffffffu, id[0]);
        if (cur == 0xffffffffu) break;
        const bool has = id[0] == cur; // ids are distinct within a pixel's set
        const float wsel = w[0];
        const int64_t kdi = pix * K + so.first();
        if (has) {
#pragma unroll
            for (int s = 0; s + 1 < KMAX; ++s) {
                id[s] = id[s + 1];
                w[s] = w[s + 1];
            }
            id[KMAX - 1] = 0xffffffffu;
            so.pop();
        }
        uint32_t m = __ballot_sync(0xffffffffu, has);
        // the surfel's feature row (dequantised), this lane's channels
        float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0;
        if (c0on) {
            f0 = load_feat4<DT>(a.feat, cur, a.D, 4 * lane);
            f0 = make_float4(f0.x * sc0.x, f0.y * sc0.y, f0.z * sc0.z, f0.w * sc0.w);
        }
        if (c1on) {
            f1 = load_feat4<DT>(a.feat, cur, a.D, 4 * lane + 128);
            f1 = make_float4(f1.x * sc1.x, f1.y * sc1.y, f1.z * sc1.z, f1.w * sc1.w);
        }
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        while (m) {
            // up to four selecting pixels per round so their gF loads overlap
            const uint32_t before = m;
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
            const uint32_t taken = before & ~m;
            float wq[4], part[4];
            float4 g0[4], g1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool on = q < nL;
                wq[q] = on ? __shfl_sync(0xffffffffu, wsel, Ls[q]) : 0.0f;
                const long long pL = __shfl_sync(0xffffffffu, static_cast<long long>(pix), Ls[q]);
                const float4 *row = reinterpret_cast<const float4 *>(a.g_F + pL * a.D);
                g0[q] = (on && c0on) ? __ldg(row + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                g1[q] = (on && c1on) ? __ldg(row + lane + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
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
                part[q] = dot4(g1[q], f1, dot4(g0[q], f0, 0.0f));
            }
            // kd of the round's pixels: lane 8q holds the q-th total
            const float tot = warp_transpose_sum4(part, lane);
            const int myq = min(__popc(taken & lt), 3);
            const float mykd = __shfl_sync(0xffffffffu, tot, 8 * myq);
            if ((taken >> lane) & 1u) a.kd[kdi] = mykd;
        }
        if (a.g_feat) {
            float4 *dst = reinterpret_cast<float4 *>(a.g_feat + static_cast<int64_t>(cur) * a.D);
            if (c0on) atomicAdd(dst + lane, acc0);
            if (c1on) atomicAdd(dst + lane + 32, acc1);
        }
    }
}

// D <= 128 and K <= 8: the warp takes its 32 pixels in two passes of 16
// (lanes 16h .. 16h + 15, the upper and lower half of its 8x4 block). A pass
// first loads the g_F rows of its 16 pixels into registers (lanes across
// channels: 16 float4 per lane, all loads in flight together), then visits
// the distinct surfels its pixels selected in ascending id; per surfel only
// the feature row is read (the next surfel's row is requested before the
// current one is used). omega gF goes into the surfel's dL/df as above; the
// 16 pixels' partial dots <gF, f> are summed by one transposing butterfly
// (one per half-row holding a selecting pixel measured slower).
// Against the per-surfel rounds above, no g_F row is read twice.
template <int DT>
__global__ void __launch_bounds__(256, 2) feat_bwd_reg_kernel(const __grid_constant__ FrameParams fp, FeatBwdArgs a)
{
    constexpr int KMAX = 8;
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

    uint32_t id[KMAX];
    float w[KMAX];
    SlotOrder<KMAX> so;
    load_sorted_set<KMAX>(fp, a, inside, pix, id, w, so);

    // lane l owns channels [4l, 4l + 4)
    const bool con = lane < (a.D >> 2);
    float4 sc = make_float4(1.f, 1.f, 1.f, 1.f);
    if (a.fscale && con) {
        const float *p = a.fscale + 4 * lane; // the scale array has no alignment beyond 4 bytes
        sc = make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), __ldg(p + 3));
    }
    auto feat_row = [&](uint32_t i) {
        if (!con || i == 0xffffffffu) return make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 f = load_feat4<DT>(a.feat, i, a.D, 4 * lane);
        return make_float4(f.x * sc.x, f.y * sc.y, f.z * sc.z, f.w * sc.w);
    };
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const bool mine_pass = (lane >> 4) == h;
        float4 G[16];
#pragma unroll
        for (int p = 0; p < 16; ++p) {
            const int src = 16 * h + p;
            const long long pL = __shfl_sync(0xffffffffu, static_cast<long long>(pix), src);
            const int inL = __shfl_sync(0xffffffffu, inside ? 1 : 0, src);
            G[p] = (inL && con) ? __ldg(reinterpret_cast<const float4 *>(a.g_F + pL * a.D) + lane)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        uint32_t cur = __reduce_min_sync(0xffffffffu, mine_pass ? id[0] : 0xffffffffu);
        float4 f = feat_row(cur);
        while (cur != 0xffffffffu) {
            const bool has = mine_pass && id[0] == cur; // ids are distinct within a pixel's set
            const float wsel = w[0];
            const long long kdi = static_cast<long long>(pix * K + so.first());
            if (has) {
#pragma unroll
                for (int s = 0; s + 1 < KMAX; ++s) {
                    id[s] = id[s + 1];
                    w[s] = w[s + 1];
                }
                id[KMAX - 1] = 0xffffffffu;
                so.pop();
            }
            const uint32_t m = __ballot_sync(0xffffffffu, has) >> (16 * h);
            const uint32_t nxt = __reduce_min_sync(0xffffffffu, mine_pass ? id[0] : 0xffffffffu);
            const float4 fn = feat_row(nxt);
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            float part[16];
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                part[p] = 0.0f;
                if ((m >> p) & 1u) {
                    const float wp = __shfl_sync(0xffffffffu, wsel, 16 * h + p);
                    // packed FMAs, two channels each
                    const float2 w2 = make_float2(wp, wp);
                    const float2 lo = __ffma2_rn(w2, make_float2(G[p].x, G[p].y), make_float2(acc.x, acc.y));
                    const float2 hi = __ffma2_rn(w2, make_float2(G[p].z, G[p].w), make_float2(acc.z, acc.w));
                    acc = make_float4(lo.x, lo.y, hi.x, hi.y);
                    const float2 d = __ffma2_rn(make_float2(G[p].z, G[p].w), make_float2(f.z, f.w),
                                                __fmul2_rn(make_float2(G[p].x, G[p].y), make_float2(f.x, f.y)));
                    part[p] = d.x + d.y;
                }
            }
            // lane l ends with the total of the pass's pixel l >> 1
            const float tot = warp_transpose_sum16(part, lane);
            const long long kdw = __shfl_sync(0xffffffffu, kdi, 16 * h + (lane >> 1));
            if ((lane & 1) == 0 && ((m >> (lane >> 1)) & 1u)) a.kd[kdw] = tot;
            if (a.g_feat && con) atomicAdd(reinterpret_cast<float4 *>(a.g_feat + static_cast<int64_t>(cur) * a.D) + lane, acc);
            cur = nxt;
            f = fn;
        }
    }
}

template <int KMAX, int NCH>
cudaError_t launch_kn(const FrameParams &fp, const FeatView &f, const FeatBwdArgs &a, cudaStream_t st)
{
    const unsigned grid = static_cast<unsigned>(fp.n_tiles_total);
    switch (f.dtype) {
    case PSI_BF16: feat_bwd_kernel<KMAX, PSI_BF16, NCH><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
    case PSI_FP8_E4M3: feat_bwd_kernel<KMAX, PSI_FP8_E4M3, NCH><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
    default: feat_bwd_kernel<KMAX, PSI_F32, NCH><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
    }
    return cudaGetLastError();
}

template <int KMAX>
cudaError_t launch_k(const FrameParams &fp, const FeatView &f, const FeatBwdArgs &a, cudaStream_t st)
{
    if (KMAX == 8 && f.dim <= 128) {
        const unsigned grid = static_cast<unsigned>(fp.n_tiles_total);
        switch (f.dtype) {
        case PSI_BF16: feat_bwd_reg_kernel<PSI_BF16><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
        case PSI_FP8_E4M3: feat_bwd_reg_kernel<PSI_FP8_E4M3><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
        default: feat_bwd_reg_kernel<PSI_F32><<<grid, 16 * fp.tile_h, 0, st>>>(fp, a); break;
        }
        return cudaGetLastError();
    }
    return f.dim > 128 ? launch_kn<KMAX, 2>(fp, f, a, st) : launch_kn<KMAX, 1>(fp, f, a, st);
}

} // namespace

cudaError_t launch_feat_bwd(const FrameParams &fp, const FeatView &f, const int32_t *topk_ids, const float *topk_w,
                            const float *g_F, float *kd, float *g_feat, DevStatus *status, cudaStream_t st)
{
    if (fp.n_tiles_total == 0 || fp.top_k <= 0 || !f.data || !g_F) return cudaSuccess;
    FeatBwdArgs a{};
    a.feat = f.data;
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
