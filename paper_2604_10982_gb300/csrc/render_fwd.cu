// a4: per-tile compositing with Top-K Hard Selection.
//
// One CTA per 16x16 tile, one thread per pixel. The tile's sorted list is
// walked in batches of 256 records staged into shared memory by TMA bulk
// copies (double buffered, mbarrier completion), so the next batch streams in
// while the current one is composited. Per pixel (Sec. 3.1, Eq. 1): alpha =
// min(0.99, o exp(-(u^2+v^2)/2)), RGB blended densely front to back with FP32
// transmittance T, and the K largest weights omega_j = alpha_j T_j kept in
// registers (Sec. 5, Top-K Hard Selection): the insertion runs under a
// warp vote, so lanes pay one compare per surfel unless some lane of the warp
// improves its set. After the walk the K selected features are gathered with
// 16-byte vector loads and summed in list order in FP32:
// F = scale * sum_{j in K} omega_j q_j.
// Dense features (K = 0) accumulate 32 channels per pass over the list.
#include "raster.cuh"

namespace psi {
namespace {

using namespace raster;

struct FwdArgs {
    const float4 *records;
    const uint32_t *vals;
    const uint32_t *ranges;
    const void *feat;
    const float *fscale;
    int D;
    bool wide; // feature rows read 32 bytes at a time
    int c0;          // dense mode: first channel of this pass
    int write_rgb;   // dense mode: only the first pass writes rgb / T / ids
    float *rgb;
    float *T;
    int32_t *n_last;
    void *F;
    int F_bf16;
    int32_t *topk_ids;
    float *topk_w;
    int32_t *argmax;
    DevStatus *status;
    unsigned int *work; // persistent launch: the context's tile counter pair; NULL: one tile per CTA
};

// One tile of the frame (the whole CTA; P freshly initialised by thread 0
// below). TH: tile height (16x16 or 16x8 tiles).
template <int KMAX, int DT, int CH, bool LP, int TH>
__device__ __forceinline__ void fwd_tile(const FrameParams &fp, const FwdArgs &a, Pipe &P, uint32_t tile)
{
    constexpr int PW = pixel_warps(TH);
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const int v = view_of_tile(fp, tile);
    const ViewParams &cam = fp.v[v];
    const int local = static_cast<int>(tile - cam.tile_base);
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
    const int64_t list0 = a.ranges[2 * tile];
    int n = static_cast<int>(a.ranges[2 * tile + 1] - a.ranges[2 * tile]);
    if (!PSI_CHECK(a.ranges[2 * tile + 1] >= a.ranges[2 * tile], kChkRange, a.status)) n = 0;
    const int nb = (n + kPB - 1) / kPB;
    const uint32_t rec_lo = static_cast<uint32_t>(static_cast<int64_t>(v) * fp.n);
    const uint32_t rec_hi = static_cast<uint32_t>(static_cast<int64_t>(v + 1) * fp.n);

    // A 16x8 tile is the upper or lower half of the 16x16 tile it lies in:
    // records are folded at that 16x16 tile's origin and its pixel warps play
    // warps 0-3 or 4-7 of it, so every pixel evaluates exactly the float32
    // sequence of the 16x16 launch (same results bit for bit).
    const int oy = (ty * TH) & 15;
    const int vw = wid + (oy ? pixel_warps(16) / 2 : 0); // warp of the 16x16 tile this warp plays
    if (tid == 0) pipe_init(P, PW);
    __syncthreads();
    if (wid == PW) {
        pipe_produce(P, a.vals, list0, n, false, a.records, tx * kTile, ty * TH - oy, a.status, kSiteRenderFwd,
                     rec_lo, rec_hi);
        return;
    }

    int lxi, lyi;
    pixel_of_thread(vw * 32 + lane, lxi, lyi);
    const int px = tx * kTile + lxi, py = ty * TH - oy + lyi;
    const bool inside = px < cam.W && py < cam.H;
    const float lx = static_cast<float>(lxi), ly = static_cast<float>(lyi);
    const int64_t surf0 = static_cast<int64_t>(v) * fp.n;
    const int K = KMAX > 0 ? fp.top_k : 0;

    float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    int last = 0;
    bool done = !inside;
    TopK<(KMAX > 0 ? KMAX : 1)> top;
    top.init(K);
    float facc[KMAX == 0 ? CH : 1];
#pragma unroll
    for (int c = 0; c < (KMAX == 0 ? CH : 1); ++c) facc[c] = 0.0f;

    bool wdone = __all_sync(0xffffffffu, done);
    if (wdone && lane == 0) atomicSub(&P.alive, 1);
    for (int b = 0; b < nb; ++b) {
        if (!pipe_wait_ready(P, b, a.status, kSiteRenderFwd)) break;
        const int st = b % kPS;
        int cnt;
        const int lo = batch_range(b, n, false, cnt);
        if (!wdone) {
            // only the records that touch this warp's pixel block, in list order
            uint32_t hw[kPB / 32];
            pipe_hit_words(P, st, cnt, vw, hw);
            bool all_done = false;
#pragma unroll 1
            for (int q = 0; q < kPB / 32 && !all_done; ++q)
#pragma unroll 1
            for (uint32_t bits = q == 0 ? hw[0] : q == 1 ? hw[1] : q == 2 ? hw[2] : hw[3]; bits; bits &= bits - 1) {
                if (__all_sync(0xffffffffu, done)) {
                    all_done = true;
                    break;
                }
                const int j = q * 32 + __ffs(bits) - 1;
                const Rec r = load_rec(P.rec[st][j]);
                Eval e;
                const bool hit = !done && eval_alpha<LP>(r, lx, ly, e);
                const float w = hit ? __fmul_rn(e.alpha, T) : 0.0f;
                const int pos = lo + j;
                if (hit) {
                    const float4 col = P.rec[st][j][3];
                    cr = __fmaf_rn(w, col.y, cr);
                    cg = __fmaf_rn(w, col.z, cg);
                    cb = __fmaf_rn(w, col.w, cb);
                    if constexpr (KMAX == 0) {
                        if (a.feat) {
                            float f[CH];
                            load_feat<DT, CH>(a.feat, static_cast<int64_t>(P.val[st][j]) - surf0, a.D, a.c0, f, a.wide);
#pragma unroll
                            for (int c = 0; c < CH; ++c) facc[c] = __fmaf_rn(w, f[c], facc[c]);
                        }
                    }
                }
                if constexpr (KMAX > 0) top.offer(hit, w, pos);
                if (hit) {
                    T = __fmul_rn(T, __fsub_rn(1.0f, e.alpha));
                    last = pos + 1;
                    if (T < fp.t_eps) done = true;
                }
            }
        }
        pipe_release(P, b);
        if (!wdone && __all_sync(0xffffffffu, done)) {
            wdone = true;
            if (lane == 0) atomicSub(&P.alive, 1);
        }
    }
    if (vload(P.abort)) return;
    if (!inside) return;

    const int64_t pix = cam.pix_base + static_cast<int64_t>(py) * cam.W + px;
    if (a.write_rgb) {
        a.rgb[pix] = cr;
        a.rgb[fp.n_pix_total + pix] = cg;
        a.rgb[2 * fp.n_pix_total + pix] = cb;
        a.T[pix] = T;
        if (a.n_last) a.n_last[pix] = last;
    }

    if constexpr (KMAX == 0) {
        if (a.F && a.feat) store_feat<CH>(a.F, a.F_bf16 != 0, pix, a.D, a.c0, facc, a.fscale);
    } else {
        top.sort_by_pos();
        int32_t sid[KMAX];
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            sid[s] = top.valid(s, K) ? static_cast<int32_t>(static_cast<int64_t>(a.vals[list0 + top.p[s]]) - surf0) : -1;
            if (!PSI_CHECK(sid[s] >= -1 && sid[s] < fp.n, kChkFeatRow, a.status)) sid[s] = -1;
        }
        if (a.topk_ids) {
            int32_t *dst = a.topk_ids + pix * K;
#pragma unroll
            for (int s = 0; s < KMAX; ++s)
                if (s < K) dst[s] = sid[s];
        }
        if (a.topk_w) {
            float *dst = a.topk_w + pix * K;
#pragma unroll
            for (int s = 0; s < KMAX; ++s)
                if (s < K) dst[s] = sid[s] >= 0 ? top.w[s] : 0.0f;
        }
        if ((a.F || a.argmax) && a.feat) {
            // 16 channels per chunk keeps the gather's registers low (one
            // 32-byte BF16 row slice = two 16-byte loads per selected surfel)
            constexpr int CB = 16;
            float best = -__int_as_float(0x7f800000);
            int arg = 0;
            for (int c0 = 0; c0 < a.D; c0 += CB) {
                float acc[CB];
#pragma unroll
                for (int c = 0; c < CB; ++c) acc[c] = 0.0f;
#pragma unroll
                for (int s = 0; s < KMAX; ++s) {
                    if (sid[s] < 0) continue;
                    float f[CB];
                    load_feat<DT, CB>(a.feat, sid[s], a.D, c0, f, a.wide);
#pragma unroll
                    for (int c = 0; c < CB; ++c) acc[c] = __fmaf_rn(top.w[s], f[c], acc[c]);
                }
                if (a.F) store_feat<CB>(a.F, a.F_bf16 != 0, pix, a.D, c0, acc, a.fscale);
                if (a.argmax) {
#pragma unroll
                    for (int c = 0; c < CB; ++c) {
                        const float val = a.fscale ? acc[c] * __ldg(a.fscale + c0 + c) : acc[c];
                        if (val > best) {
                            best = val;
                            arg = c0 + c;
                        }
                    }
                }
            }
            if (a.argmax) a.argmax[pix] = (1.0f - T < 1e-4f) ? -1 : arg;
        }
    }
}

// OCC: CTAs per SM the kernel is built for (the launch shape the autotuner
// picks). Tiles are taken longest list first: CTA b starts with entry b of the
// launch order; in the persistent launch (a.work set, grid of a few CTAs per
// SM) each CTA then fetches the next entry from the context's counter until
// the order is exhausted, and the last CTA to finish resets the counter pair
// for the next launch (launches through one context must not overlap).
template <int KMAX, int DT, int CH, bool LP, int OCC, int TH = 16>
__global__ void __launch_bounds__(pipe_threads(TH), OCC)
    render_fwd_kernel(const __grid_constant__ FrameParams fp, FwdArgs a)
{
    __shared__ __align__(128) Pipe P;
    __shared__ uint32_t s_next;
    uint32_t i = blockIdx.x;
    while (true) {
        const uint32_t tile = a.ranges[2 * fp.n_tiles_total + i];
        // debug builds: the launch order must name a tile of the frame (uniform for the CTA)
        if (PSI_CHECK(tile < fp.n_tiles_total, kChkTile, a.status)) fwd_tile<KMAX, DT, CH, LP, TH>(fp, a, P, tile);
        if (!a.work) break;
        __syncthreads(); // every warp is done with this tile's pipeline
        if (threadIdx.x == 0) {
            s_next = vload(P.abort) ? 0xffffffffu : gridDim.x + atomicAdd(&a.work[0], 1u);
            pipe_inval(P);
        }
        __syncthreads();
        i = s_next;
        if (i >= fp.n_tiles_total) break;
    }
    if (a.work && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&a.work[1], 1u) == gridDim.x - 1) {
            a.work[0] = 0u;
            a.work[1] = 0u;
        }
    }
}

template <int KMAX, int CH, bool LP, int OCC, int TH = 16>
cudaError_t launch_kclo(const FrameParams &fp, const FeatView &f, const FwdArgs &a, cudaStream_t st)
{
    unsigned grid = fp.n_tiles_total;
    if (a.work) grid = persistent_grid(fp.n_tiles_total, OCC);
    constexpr int nt = pipe_threads(TH);
    switch (f.data ? f.dtype : PSI_F32) {
    case PSI_BF16: render_fwd_kernel<KMAX, PSI_BF16, CH, LP, OCC, TH><<<grid, nt, 0, st>>>(fp, a); break;
    case PSI_FP8_E4M3: render_fwd_kernel<KMAX, PSI_FP8_E4M3, CH, LP, OCC, TH><<<grid, nt, 0, st>>>(fp, a); break;
    default: render_fwd_kernel<KMAX, PSI_F32, CH, LP, OCC, TH><<<grid, nt, 0, st>>>(fp, a); break;
    }
    return cudaGetLastError();
}

// 16x8 tiles (Top-K with K <= 8, no low-pass filter): 4 pixel warps, up to 5 CTAs per SM
constexpr int kOccTile8 = 5;

template <int KMAX, int CH, bool LP>
cudaError_t launch_kcl(const FrameParams &fp, const FeatView &f, const FwdArgs &a, bool alt, cudaStream_t st)
{
    // K <= 8: 3 CTAs per SM (4 as the alternative); larger K and dense: 2 (1)
    constexpr int occ = (KMAX > 0 && KMAX <= 8) ? 3 : 2;
    constexpr int occ_alt = (KMAX > 0 && KMAX <= 8) ? 4 : 1;
    return alt ? launch_kclo<KMAX, CH, LP, occ_alt>(fp, f, a, st) : launch_kclo<KMAX, CH, LP, occ>(fp, f, a, st);
}

template <int KMAX, int CH>
cudaError_t launch_kc(const FrameParams &fp, const FeatView &f, const FwdArgs &a, bool alt, cudaStream_t st)
{
    return fp.lowpass ? launch_kcl<KMAX, CH, true>(fp, f, a, alt, st) : launch_kcl<KMAX, CH, false>(fp, f, a, alt, st);
}

template <int KMAX>
cudaError_t launch_k(const FrameParams &fp, const FeatView &f, const FwdArgs &a, int ch, bool alt, cudaStream_t st)
{
    if (fp.n_tiles_total == 0) return cudaSuccess;
    // the channel chunk only shapes the dense (K = 0) accumulation
    if constexpr (KMAX > 0)
        return launch_kc<KMAX, 16>(fp, f, a, alt, st);
    else
        return ch == 32 ? launch_kc<KMAX, 32>(fp, f, a, alt, st) : launch_kc<KMAX, 16>(fp, f, a, alt, st);
}

} // namespace

cudaError_t launch_render_fwd(const FrameParams &fp, const FeatView &f, const float4 *records, const uint32_t *vals,
                              const uint32_t *ranges, const psi_fwd_out &out, DevStatus *status, cudaStream_t st,
                              int shape)
{
    FwdArgs a{};
    a.records = records;
    a.vals = vals;
    a.ranges = ranges;
    a.feat = f.data;
    a.wide = f.data && feat_rows_wide(f.data, f.dim, f.dtype);
    a.fscale = f.scale;
    a.D = f.dim;
    a.c0 = 0;
    a.write_rgb = 1;
    a.rgb = out.rgb;
    a.T = out.T;
    a.n_last = out.n_last;
    a.F = out.F;
    a.F_bf16 = out.F_dtype == PSI_BF16;
    a.topk_ids = out.topk_ids;
    a.topk_w = out.topk_w;
    a.argmax = out.argmax;
    a.status = status;
    const int K = fp.top_k;
    const int ch = render_channel_chunk(f.dim, K, shape);
    const bool alt = shape & kShapeAltOcc;
    a.work = (shape & kShapePersistent) ? status->work : nullptr;
    if (K == 0) {
        // dense: one pass per chunk of channels (the first also writes rgb/T)
        cudaError_t e = launch_k<0>(fp, f, a, ch, alt, st);
        for (int c0 = ch; e == cudaSuccess && f.data && out.F && c0 < f.dim; c0 += ch) {
            a.c0 = c0;
            a.write_rgb = 0;
            e = launch_k<0>(fp, f, a, ch, alt, st);
        }
        return e;
    }
    if (fp.tile_h == 8) return launch_kclo<8, 16, false, kOccTile8, 8>(fp, f, a, st);
    if (K <= 8) return launch_k<8>(fp, f, a, ch, alt, st);
    if (K <= 16) return launch_k<16>(fp, f, a, ch, alt, st);
    return launch_k<32>(fp, f, a, ch, alt, st);
}

} // namespace psi
