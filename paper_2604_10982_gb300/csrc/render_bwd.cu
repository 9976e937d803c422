// a5: adjoint of the per-tile compositing with Top-K Hard Selection.
//
// Pass A recomputes the forward walk of each pixel with the same float32
// operation sequence (shared eval_alpha and TopK helpers), which recovers the
// same Top-K set, T_final and last surfel without storing per-pixel lists.
// Pass B walks the tile's list back to front. With C = sum_j c_j alpha_j T_j
// (Eq. 1), F = sum_{j in K} f_j omega_j (Sec. 5) and
// L = <gC, C> + <gF, F> + gT T_final:
//     s_j        = <gC, c_j> + [j in K] <gF, f_j>
//     dL/dalpha_j = T_j s_j - (sum_{k>j} omega_k s_k + T_final gT) / (1 - alpha_j)
//     dL/dc_j    += omega_j gC,     dL/df_j += [j in K] omega_j gF
// T_j is recovered as T_{j+1} / (1 - alpha_j). Through alpha = o G (unless
// clamped): dL/do = dL/dalpha G, and (u, v) enter via a = dL/dalpha * alpha:
// with (u, v, 1) ~ M^-1 p the gradient of M is M^-T W, W = sum a (u, v,
// -d^2)(u, v, 1)^T, so each (pixel, record) adds 7 moments of (u, v).
// Per-record sums (colour, dL/do, moments) go to a per-record slot array:
// when at most twelve lanes of the warp contribute, each adds its 11 values with
// three 16-byte vector reductions; otherwise they are reduced across the warp
// (a transposing butterfly: 11 values in 13 shuffles) and added with one
// atomic per value per warp. The feature gradient is accumulated
// warp-cooperatively across channels.
// With the 2DGS low-pass filter, a pixel where the screen-space term
// rho = 2 |x - p0|^2 wins adds dL/dp0 = 2 a (x - p0) (a = dL/dalpha * alpha)
// instead of the (u, v) moments: 13 sums (16-slot butterfly, 16 shuffles)
// and two more moments per record, taken through the projection of mu.
// Both passes stream the list through the same producer-warp pipeline as the
// forward kernel (raster.cuh): pass A front to back until every pixel is
// saturated, pass B back to front from the largest last-composited position
// of the tile; a warp visits only the records that meet its 8x4 block, and in
// pass B only those before the last surfel of one of its pixels.
// With the forward's saved state and a Top-K selection, pass B also exists
// in a form with two pixels per lane (bwd_tile_pair below; a launch shape).
// A second kernel turns the per-record moments into gradients of mu, t_u,
// t_v, s_u, s_v through the camera.
#include "raster.cuh"

namespace psi {
namespace {

using namespace raster;

// per record: dL/dc (3), dL/do, Suu, Suv, Svv, Su, Sv, Sdu, Sdv, padding; with
// the low-pass filter also dL/dp0x, dL/dp0y and three padding floats -- whole
// float4s, so that a pixel can add its share with 16-byte vector reductions
__host__ __device__ constexpr int moments_per_record(bool lp) { return lp ? 16 : 12; }

struct BwdArgs {
    const float4 *records;
    const uint32_t *vals;
    const uint32_t *ranges;
    const void *feat;
    const float *fscale;
    int D;
    bool wide; // feature rows read 32 bytes at a time
    const float *g_rgb; // [3][P_total]
    const float *g_F;   // [P_total, D] or NULL
    const float *g_T;   // [P_total] or NULL
    float *g_feat;      // [N,D] or NULL
    float *moments;     // [R, moments_per_record]
    DevStatus *status;
    // forward state of the same frame (all NULL: recompute it in pass A)
    const float *saved_T;      // [P_total]
    const int32_t *saved_last; // [P_total]
    const int32_t *saved_topk; // [P_total, K] surfel ids in list order, -1 padded
    const float *kd_saved;     // [P_total, K] <gF, f_j> of the saved set (feat_bwd.cu), or NULL
    unsigned int *work;        // persistent launch: the context's adjoint tile counter pair; NULL: one tile per CTA
};

// Sum 12 per-lane values over the warp (a transposing butterfly, 13
// shuffles): afterwards lane l (and l ^ 1) holds the total of value index
// 6 b4 + 3 b3 + g with g = 2 b2 + b1 (b_k = bit k of l); lanes with g = 3 hold
// a padding slot.
__device__ __forceinline__ float warp_transpose_sum12(float v[12], int lane)
{
#pragma unroll
    for (int k = 0; k < 6; ++k) { // 12 -> 6: halves [0, 6) / [6, 12)
        const bool hi = lane & 16;
        const float send = hi ? v[k] : v[k + 6];
        const float keep = hi ? v[k + 6] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) { // 6 -> 3
        const bool hi = lane & 8;
        const float send = hi ? v[k] : v[k + 3];
        const float keep = hi ? v[k + 3] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    v[3] = 0.0f; // 3 -> 4 slots (one padding)
#pragma unroll
    for (int k = 0; k < 2; ++k) { // 4 -> 2
        const bool hi = lane & 4;
        const float send = hi ? v[k] : v[k + 2];
        const float keep = hi ? v[k + 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2; // 2 -> 1
        const float send = hi ? v[0] : v[1];
        const float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// The saved Top-K set of one pixel met during pass B. The saved ids are in
// list order, so walking back to front the next selected surfel the pixel
// meets is always the last of its set not met yet: one compare per (record,
// pixel). Keeps that id and its <gF, f>, the one after it (prefetched when
// one is met, so its load has a whole stretch of the walk to land) and the
// slot before that.
struct SavedSel {
    int nid, nnid, ptr;
    float nkd, nnkd;

    __device__ __forceinline__ void init(const BwdArgs &a, int64_t pix, int K, int64_t n_surf, bool on)
    {
        nid = nnid = ptr = -1;
        nkd = nnkd = 0.0f;
        if (!on || !a.kd_saved) return;
        const int32_t *ids = a.saved_topk + pix * K;
        const float *kds = a.kd_saved + pix * K;
#pragma unroll 4
        for (int s = 0; s < K; ++s) {
            int id = ids[s];
            // debug builds: a saved id must be -1 or a surfel of the table
            if (!PSI_CHECK(id >= -1 && id < n_surf, kChkFeatRow, a.status)) id = -1;
            if (id >= 0) {
                nnid = nid;
                nnkd = nkd;
                nid = id;
                nkd = kds[s];
                ptr = s - 2;
            }
        }
    }

    // <gF, f_sid> if sid is the pixel's next selected surfel (then advance), else 0
    __device__ __forceinline__ float match(const BwdArgs &a, int64_t pix, int K, int64_t n_surf, int sid)
    {
        if (sid != nid) return 0.0f;
        const float dot = nkd;
        nid = nnid;
        nkd = nnkd;
        nnid = -1;
        nnkd = 0.0f;
        if (ptr >= 0) {
            int id = a.saved_topk[pix * K + ptr];
            if (!PSI_CHECK(id >= -1 && id < n_surf, kChkFeatRow, a.status)) id = -1;
            nnid = id;
            nnkd = a.kd_saved[pix * K + ptr];
        }
        --ptr;
        return dot;
    }
};

// Up to this many contributing lanes add their values with their own 16-byte
// vector reductions (3 or 4 per lane) instead of reducing over the warp first:
// the walk is bound by instruction issue and the L2 has atomic throughput to
// spare, so the reductions pay off up to 12-16 lanes (1.61 ms for the walk of
// the 3M-surfel frame at 12, against 1.70 at 4, 1.67 at 20, 3.06 at 32).
constexpr int kDirectLanes = 12;

// Adds one record's per-lane sums (the lane contributes if `act`) to its
// 16-byte aligned slot array: by direct vector reductions up to kDirectLanes
// contributing lanes, else through the warp butterfly and one atomic per sum.
// (Adding lane pairs first and reducing directly from the even lanes up to 24
// or 32 contributing lanes measured slower: 1.64 and 1.90 ms against 1.58 ms
// for the walk of the 3M-surfel frame.)
template <bool LP>
__device__ __forceinline__ void add_record_sums(float *vals, bool act, uint32_t amask, int lane, float *slots)
{
    constexpr int kM = moments_per_record(LP);
    constexpr int kSums = LP ? 13 : 11;
    if (__popc(amask) <= kDirectLanes) {
        if (act) {
            float4 *dst = reinterpret_cast<float4 *>(slots);
#pragma unroll
            for (int k4 = 0; k4 < kM / 4; ++k4)
                atomicAdd(dst + k4, make_float4(vals[4 * k4], vals[4 * k4 + 1], vals[4 * k4 + 2], vals[4 * k4 + 3]));
        }
        return;
    }
    float tot;
    int idx;
    bool mine;
    if constexpr (LP) {
        tot = warp_transpose_sum16(vals, lane);
        idx = (lane >> 1) & 15;
        mine = (lane & 1) == 0 && idx < kSums;
    } else {
        tot = warp_transpose_sum12(vals, lane);
        const int g = ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
        idx = ((lane >> 4) & 1) * 6 + ((lane >> 3) & 1) * 3 + g;
        mine = (lane & 1) == 0 && g < 3;
    }
    if (mine && tot != 0.0f) atomicAdd(slots + idx, tot);
}

// SAVED: T_final, last and the Top-K ids come from the forward's outputs;
// otherwise pass A recomputes them. With SAVED and K > 0 the feature terms
// (<gF, f_j> and dL/df) come from the per-pixel feature kernel instead of this
// walk. CH (channel chunk) matters only for K = 0.
// One tile (the whole CTA; P freshly initialised by thread 0 below).
// NW (dense features with D = 16, e.g. the depth/normal table): each pixel's
// g_F row is held in registers for the whole walk, and dL/df of a record is
// summed over the warp by one 16-value transposing butterfly (one atomic per
// channel) instead of the lanes-across-channels rounds, which would leave 28
// of 32 lanes idle at 16 channels.
template <int KMAX, int DT, int CH, bool SAVED, bool LP, int TH, bool NW = false>
__device__ __forceinline__ void bwd_tile(const FrameParams &fp, const BwdArgs &a, Pipe &P, int &s_maxlast,
                                         uint32_t tile)
{
    constexpr int PW = pixel_warps(TH);
    constexpr int kM = moments_per_record(LP);
    constexpr int kSlots = LP ? 16 : 12;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const bool producer = wid == PW;
    const int v = view_of_tile(fp, tile);
    const ViewParams &cam = fp.v[v];
    const int local = static_cast<int>(tile - cam.tile_base);
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
    const int64_t list0 = a.ranges[2 * tile];
    int n = static_cast<int>(a.ranges[2 * tile + 1] - a.ranges[2 * tile]);
    if (!PSI_CHECK(a.ranges[2 * tile + 1] >= a.ranges[2 * tile], kChkRange, a.status)) n = 0;
    const int64_t surf0 = static_cast<int64_t>(v) * fp.n;
    const uint32_t rec_lo = static_cast<uint32_t>(surf0);
    const uint32_t rec_hi = static_cast<uint32_t>(surf0 + fp.n);
    const int K = KMAX > 0 ? fp.top_k : 0;
    // a 16x8 tile plays the upper or lower half of its 16x16 tile (see the
    // forward kernel): same folded records, same per-pixel float32 sequence
    const int oy = (ty * TH) & 15;
    const int vw = wid + (oy ? pixel_warps(16) / 2 : 0);
    const int tileX = tx * kTile, tileY = ty * TH - oy;
    int lxi = 0, lyi = 0;
    if (!producer) pixel_of_thread(vw * 32 + lane, lxi, lyi);
    const int px = tileX + lxi, py = tileY + lyi;
    const bool inside = !producer && px < cam.W && py < cam.H;
    const float lx = static_cast<float>(lxi), ly = static_cast<float>(lyi);
    const int64_t pix = cam.pix_base + static_cast<int64_t>(min(py, cam.H - 1)) * cam.W + min(px, cam.W - 1);

    if (tid == 0) {
        pipe_init(P, PW);
        s_maxlast = 0;
    }
    __syncthreads();

    // ---------------- pass A: forward recompute (Top-K set, T_final, last),
    // unless the forward's own outputs for this frame are given
    constexpr bool recompute = !SAVED;
    constexpr bool ext_feat = SAVED && KMAX > 0; // feature terms computed outside the walk
    float T = 1.0f;
    int last = 0;
    bool done = !inside;
    TopK<(KMAX > 0 ? KMAX : 1)> top;
    top.init(K);
    if constexpr (SAVED) {
        if (inside) {
            T = a.saved_T[pix];
            last = a.saved_last[pix];
        }
        // a saved last position lies within the tile's list (it bounds the walk)
        if (!PSI_CHECK(last >= 0 && last <= n, kChkLast, a.status)) last = 0;
        last = min(max(last, 0), n);
    } else if (producer) {
        pipe_produce(P, a.vals, list0, n, false, a.records, tileX, tileY, a.status, kSiteRenderBwdA, rec_lo, rec_hi);
    } else {
        const int nb = (n + kPB - 1) / kPB;
        bool wdone = __all_sync(0xffffffffu, done);
        if (wdone && lane == 0) atomicSub(&P.alive, 1);
        for (int b = 0; b < nb; ++b) {
            if (!pipe_wait_ready(P, b, a.status, kSiteRenderBwdA)) break;
            const int st = b % kPS;
            int cnt;
            const int lo = batch_range(b, n, false, cnt);
            if (!wdone) {
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
                    if constexpr (KMAX > 0) top.offer(hit, w, lo + j);
                    if (hit) {
                        T = __fmul_rn(T, __fsub_rn(1.0f, e.alpha));
                        last = lo + j + 1;
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
    }

    // selected set (surfel ids; a surfel occurs at most once in a tile's list)
    // and <gF, f_j> for each selected surfel
    float kd[KMAX > 0 ? KMAX : 1];
    int kid[KMAX > 0 ? KMAX : 1];
    SavedSel sel_saved; // the saved set (ext_feat), met in reverse list order
    if constexpr (KMAX > 0) {
        if constexpr (recompute) {
            top.sort_by_pos();
#pragma unroll
            for (int s = 0; s < KMAX; ++s)
            {
                kid[s] = (inside && top.valid(s, K))
                             ? static_cast<int>(static_cast<int64_t>(a.vals[list0 + top.p[s]]) - surf0)
                             : -1;
                if (!PSI_CHECK(kid[s] >= -1 && kid[s] < fp.n, kChkFeatRow, a.status)) kid[s] = -1;
            }
        }
#pragma unroll
        for (int s = 0; s < KMAX; ++s) kd[s] = 0.0f;
        if (ext_feat) {
            sel_saved.init(a, pix, K, fp.n, inside);
        } else if (a.g_F && a.feat && inside) {
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
                    if (kid[s] < 0) continue;
                    float f[16];
                    load_feat<DT, 16>(a.feat, kid[s], a.D, c0, f, a.wide);
                    float acc = kd[s];
#pragma unroll
                    for (int c = 0; c < 16; ++c) acc = __fmaf_rn(g[c], f[c], acc);
                    kd[s] = acc;
                }
            }
        }
    }
    if (inside && last > 0) atomicMax(&s_maxlast, last);
    __syncthreads(); // pass A is over for every warp and the producer drained its copies
    if constexpr (recompute) {
        if (vload(P.abort)) return;
        if (tid == 0) {
            // fresh barriers for the reverse walk
            for (int s = 0; s < kPS; ++s) {
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&P.full[s])) : "memory");
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&P.ready[s])) : "memory");
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&P.empty[s])) : "memory");
            }
            pipe_init(P, PW);
        }
        __syncthreads();
    }
    const int maxlast = s_maxlast;
    if (producer) {
        pipe_produce(P, a.vals, list0, maxlast, true, a.records, tileX, tileY, a.status, kSiteRenderBwdB, rec_lo,
                     rec_hi);
        return;
    }
    // entries at or beyond every lane's last composited surfel are skipped by the warp
    int warp_last = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) warp_last = max(warp_last, __shfl_xor_sync(0xffffffffu, warp_last, o));

    // ---------------- pass B: back to front
    const float gr = inside ? a.g_rgb[pix] : 0.0f;
    const float gg = inside ? a.g_rgb[fp.n_pix_total + pix] : 0.0f;
    const float gb = inside ? a.g_rgb[2 * fp.n_pix_total + pix] : 0.0f;
    const float gt = (inside && a.g_T) ? a.g_T[pix] : 0.0f;
    // NW: the pixel's g_F row
    float gfr[NW ? 16 : 1];
    if constexpr (NW) {
#pragma unroll
        for (int c = 0; c < 16; ++c) gfr[c] = (inside && a.g_F) ? __ldg(a.g_F + pix * 16 + c) : 0.0f;
    }
    float Tc = T;                    // T after the current surfel, walking back
    float suffix = __fmul_rn(T, gt); // sum_{k>j} omega_k s_k + T_final gT
    const int nbB = (maxlast + kPB - 1) / kPB;
    const bool want_feat = !ext_feat && a.g_F && a.g_feat;
    for (int b = 0; b < nbB; ++b) {
        if (!pipe_wait_ready(P, b, a.status, kSiteRenderBwdB)) break;
        const int st = b % kPS;
        int cnt;
        const int lo = batch_range(b, maxlast, true, cnt);
        const int limit = min(cnt, warp_last - lo); // entries [0, limit) of the batch can matter
        if (limit > 0) {
            uint32_t hw[kPB / 32];
            pipe_hit_words(P, st, cnt, vw, hw);
#pragma unroll 1
            for (int q = kPB / 32 - 1; q >= 0; --q) {
                uint32_t bits = q == 0 ? hw[0] : q == 1 ? hw[1] : q == 2 ? hw[2] : hw[3];
                const int room = limit - q * 32;
                if (room <= 0) continue;
                if (room < 32) bits &= (1u << room) - 1u;
#pragma unroll 1
                for (; bits; ) {
                    const int jj = 31 - __clz(bits);
                    bits &= ~(1u << jj);
                    const int j = q * 32 + jj;
                    const int pos = lo + j;
                    const Rec r = load_rec(P.rec[st][j]);
                    Eval e;
                    const bool act = inside && pos < last && eval_alpha<LP>(r, lx, ly, e);
                    const uint32_t amask = __ballot_sync(0xffffffffu, act);
                    if (!amask) continue;
                    const uint32_t rid = P.val[st][j];
                    const int64_t sid = static_cast<int64_t>(rid) - surf0;
                    float vals[kSlots];
#pragma unroll
                    for (int k2 = 0; k2 < kSlots; ++k2) vals[k2] = 0.0f;
                    float w = 0.0f;
                    bool sel = false;
                    if (act) {
                        const float one_m = __fsub_rn(1.0f, e.alpha);
                        const float inv = rcp_approx(one_m); // one_m >= 0.01
                        const float Tj = Tc * inv;
                        w = e.alpha * Tj;
                        float dot = 0.0f;
                        if constexpr (ext_feat) {
                            dot = sel_saved.match(a, pix, K, fp.n, static_cast<int>(sid));
                        } else if constexpr (KMAX > 0) {
#pragma unroll
                            for (int s = 0; s < KMAX; ++s)
                                if (kid[s] == static_cast<int>(sid)) {
                                    sel = true;
                                    dot = kd[s];
                                }
                        } else if (NW && a.g_F && a.feat) {
                            sel = true;
                            float f[16];
                            load_feat<DT, 16>(a.feat, sid, 16, 0, f, a.wide);
                            if (a.fscale) {
#pragma unroll
                                for (int c = 0; c < 16; ++c) dot = fmaf(gfr[c] * __ldg(a.fscale + c), f[c], dot);
                            } else {
#pragma unroll
                                for (int c = 0; c < 16; ++c) dot = fmaf(gfr[c], f[c], dot);
                            }
                        } else if (a.g_F && a.feat) {
                            // dense features: every composited surfel is selected
                            sel = true;
                            for (int c0 = 0; c0 < a.D; c0 += CH) {
                                float f[CH];
                                load_feat<DT, CH>(a.feat, sid, a.D, c0, f, a.wide);
#pragma unroll
                                for (int c = 0; c < CH; ++c) {
                                    const float sc = a.fscale ? __ldg(a.fscale + c0 + c) : 1.0f;
                                    dot = fmaf(__ldg(a.g_F + pix * a.D + c0 + c) * sc, f[c], dot);
                                }
                            }
                        }
                        const float4 col = P.rec[st][j][3];
                        const float sj = gr * col.y + gg * col.z + gb * col.w + dot;
                        const float dLda = Tj * sj - suffix * inv;
                        suffix = fmaf(w, sj, suffix);
                        Tc = Tj;
                        // products in pairs where they share a factor (packed
                        // multiplies, each rounded as the scalar one)
                        const float2 c01 = __fmul2_rn(make_float2(w, w), make_float2(gr, gg));
                        vals[0] = c01.x;
                        vals[1] = c01.y;
                        vals[2] = w * gb;
                        if (LP && !e.clamped && e.filt) {
                            // rho = 2 |x - p0|^2: dL/dp0 = (-a / 2)(-4 (x - p0))
                            const float aa = dLda * e.alpha;
                            vals[3] = dLda * e.G;
                            vals[kSlots > 12 ? 11 : 0] = 2.0f * aa * e.dx;
                            vals[kSlots > 12 ? 12 : 0] = 2.0f * aa * e.dy;
                        } else if (!e.clamped) {
                            const float rq = rcp_approx(e.q2);
                            const float2 uv = __fmul2_rn(make_float2(e.q0, e.q1), make_float2(rq, rq)); // (u, v)
                            const float d2 = uv.x * uv.x + uv.y * uv.y;
                            const float aa = dLda * e.alpha;
                            vals[3] = dLda * e.G;
                            const float2 t = __fmul2_rn(make_float2(aa, aa), uv);          // a (u, v)
                            const float2 tu = __fmul2_rn(make_float2(t.x, t.x), uv);       // a u (u, v)
                            const float ad = aa * d2;
                            const float2 td = __fmul2_rn(make_float2(ad, ad), uv);         // a d^2 (u, v)
                            vals[4] = tu.x;
                            vals[5] = tu.y;
                            vals[6] = t.y * uv.y;
                            vals[7] = t.x;
                            vals[8] = t.y;
                            vals[9] = td.x;
                            vals[10] = td.y;
                        }
                    }
                    add_record_sums<LP>(vals, act, amask, lane, a.moments + static_cast<int64_t>(rid) * kM);
                    if (NW && want_feat) {
                        if (__any_sync(0xffffffffu, act && sel)) {
                            float v[16];
#pragma unroll
                            for (int c = 0; c < 16; ++c) v[c] = (act && sel) ? w * gfr[c] : 0.0f;
                            // lane l ends with the total of channel l >> 1
                            const float tot = warp_transpose_sum16(v, lane);
                            if ((lane & 1) == 0 && tot != 0.0f) atomicAdd(a.g_feat + sid * 16 + (lane >> 1), tot);
                        }
                    } else if (want_feat) {
                        uint32_t selmask = __ballot_sync(0xffffffffu, act && sel);
                        if (selmask) {
                            // lane l owns channels [4l, 4l+4) (+128 for D=256) of the surfel's
                            // feature gradient; up to four selecting pixels per round so
                            // their g_F loads are in flight together
                            const int nv = a.D >> 2; // float4 chunks per row
                            float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
                            while (selmask) {
                                int Ls[4];
                                int nL = 0;
#pragma unroll
                                for (int qq = 0; qq < 4; ++qq) {
                                    Ls[qq] = selmask ? __ffs(selmask) - 1 : -1;
                                    if (selmask) {
                                        selmask &= selmask - 1;
                                        ++nL;
                                    }
                                }
                                float wq[4];
                                float4 g0[4], g1[4];
#pragma unroll
                                for (int qq = 0; qq < 4; ++qq) {
                                    const int L = Ls[qq] < 0 ? 0 : Ls[qq];
                                    wq[qq] = __shfl_sync(0xffffffffu, w, L);
                                    const int pL = __shfl_sync(0xffffffffu, static_cast<int>(pix), L);
                                    const float4 *grow = reinterpret_cast<const float4 *>(a.g_F + static_cast<int64_t>(pL) * a.D);
                                    const bool on = qq < nL;
                                    g0[qq] = (on && lane < nv) ? __ldg(grow + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                                    g1[qq] = (on && lane + 32 < nv) ? __ldg(grow + lane + 32) : make_float4(0.f, 0.f, 0.f, 0.f);
                                    if (!on) wq[qq] = 0.0f;
                                }
#pragma unroll
                                for (int qq = 0; qq < 4; ++qq) {
                                    acc0.x = fmaf(wq[qq], g0[qq].x, acc0.x);
                                    acc0.y = fmaf(wq[qq], g0[qq].y, acc0.y);
                                    acc0.z = fmaf(wq[qq], g0[qq].z, acc0.z);
                                    acc0.w = fmaf(wq[qq], g0[qq].w, acc0.w);
                                    acc1.x = fmaf(wq[qq], g1[qq].x, acc1.x);
                                    acc1.y = fmaf(wq[qq], g1[qq].y, acc1.y);
                                    acc1.z = fmaf(wq[qq], g1[qq].z, acc1.z);
                                    acc1.w = fmaf(wq[qq], g1[qq].w, acc1.w);
                                }
                            }
                            float4 *dst = reinterpret_cast<float4 *>(a.g_feat + sid * a.D);
                            if (lane < nv) atomicAdd(dst + lane, acc0);
                            if (lane + 32 < nv) atomicAdd(dst + lane + 32, acc1);
                        }
                    }
                }
            }
        }
        pipe_release(P, b);
    }
}

// Pixel warps of the paired walk: one 8x8 block each (two pixels per lane).
__host__ __device__ constexpr int pair_warps(int TH) { return TH / 4; }
__host__ __device__ constexpr int pair_threads(int TH) { return 32 * (pair_warps(TH) + 1); }

// Pass B from the forward's saved state with a Top-K selection (the feature
// terms <gF, f_j> come from the per-pixel feature kernel): two pixels per
// lane. A pixel warp covers an 8x8 block, rows ly and ly + 4 in each lane
// (two of the 8x4 blocks of the record masks), so the per-record work that
// does not depend on the pixel -- the staged record's loads, the vote, the
// cross-lane reduction and its atomics -- is paid once for 64 pixels; a lane
// adds its two pixels' values before the reduction.
// The saved set is matched as in the one-pixel walk (SavedSel).
template <bool LP, int TH>
__device__ __forceinline__ void bwd_tile_pair(const FrameParams &fp, const BwdArgs &a, Pipe &P, int &s_maxlast,
                                              uint32_t tile)
{
    constexpr int PW = pair_warps(TH);
    constexpr int kM = moments_per_record(LP);
    constexpr int kSlots = LP ? 16 : 12;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    const bool producer = wid == PW;
    const int v = view_of_tile(fp, tile);
    const ViewParams &cam = fp.v[v];
    const int local = static_cast<int>(tile - cam.tile_base);
    const int tx = local % cam.tiles_x, ty = local / cam.tiles_x;
    const int64_t list0 = a.ranges[2 * tile];
    int n = static_cast<int>(a.ranges[2 * tile + 1] - a.ranges[2 * tile]);
    if (!PSI_CHECK(a.ranges[2 * tile + 1] >= a.ranges[2 * tile], kChkRange, a.status)) n = 0;
    const int64_t surf0 = static_cast<int64_t>(v) * fp.n;
    const uint32_t rec_lo = static_cast<uint32_t>(surf0);
    const uint32_t rec_hi = static_cast<uint32_t>(surf0 + fp.n);
    const int K = fp.top_k;
    // a 16x8 tile plays the upper or lower half of its 16x16 tile (records are
    // folded to the 16x16 origin, as in the forward kernel)
    const int oy = (ty * TH) & 15;
    const int tileX = tx * kTile, tileY = ty * TH - oy;
    const int y0 = oy + 8 * (wid >> 1);        // first row of the warp's 8x8 block
    const int blk = (y0 >> 2) * 2 + (wid & 1); // its upper 8x4 mask block; the lower one is blk + 2
    const int lxi = (wid & 1) * 8 + (lane & 7);
    const float lx = static_cast<float>(lxi);

    if (tid == 0) {
        pipe_init(P, PW);
        s_maxlast = 0;
    }
    __syncthreads();

    float ly[2], Tc[2], suffix[2], gr[2], gg[2], gb[2];
    int last[2];
    int64_t pix[2];
    SavedSel sel[2]; // each pixel's saved set, met in reverse list order
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int lyi = y0 + (lane >> 3) + 4 * h;
        ly[h] = static_cast<float>(lyi);
        const int px = tileX + lxi, py = tileY + lyi;
        const bool inside = !producer && px < cam.W && py < cam.H;
        pix[h] = cam.pix_base + static_cast<int64_t>(min(py, cam.H - 1)) * cam.W + min(px, cam.W - 1);
        float T = 1.0f;
        int l = 0;
        if (inside) {
            T = a.saved_T[pix[h]];
            l = a.saved_last[pix[h]];
        }
        // a saved last position lies within the tile's list (it bounds the walk)
        if (!PSI_CHECK(l >= 0 && l <= n, kChkLast, a.status)) l = 0;
        last[h] = min(max(l, 0), n);
        Tc[h] = T;
        sel[h].init(a, pix[h], K, fp.n, inside);
        gr[h] = inside ? a.g_rgb[pix[h]] : 0.0f;
        gg[h] = inside ? a.g_rgb[fp.n_pix_total + pix[h]] : 0.0f;
        gb[h] = inside ? a.g_rgb[2 * fp.n_pix_total + pix[h]] : 0.0f;
        const float gt = (inside && a.g_T) ? a.g_T[pix[h]] : 0.0f;
        suffix[h] = __fmul_rn(T, gt); // sum_{k>j} omega_k s_k + T_final gT
    }
    // entries at or beyond every pixel's last composited surfel are skipped by the warp
    int warp_last = max(last[0], last[1]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) warp_last = max(warp_last, __shfl_xor_sync(0xffffffffu, warp_last, o));
    if (!producer && lane == 0 && warp_last > 0) atomicMax(&s_maxlast, warp_last);
    __syncthreads();
    const int maxlast = s_maxlast;
    if (producer) {
        pipe_produce(P, a.vals, list0, maxlast, true, a.records, tileX, tileY, a.status, kSiteRenderBwdB, rec_lo,
                     rec_hi);
        return;
    }

    const int nbB = (maxlast + kPB - 1) / kPB;
    for (int b = 0; b < nbB; ++b) {
        if (!pipe_wait_ready(P, b, a.status, kSiteRenderBwdB)) break;
        const int st = b % kPS;
        int cnt;
        const int lo = batch_range(b, maxlast, true, cnt);
        const int limit = min(cnt, warp_last - lo); // entries [0, limit) of the batch can matter
        if (limit > 0) {
            uint32_t hw[kPB / 32];
#pragma unroll
            for (int q = 0; q < kPB / 32; ++q) {
                const int j = q * 32 + lane;
                hw[q] = __ballot_sync(0xffffffffu, j < cnt && ((__float_as_uint(P.rec[st][j][4].z) >> blk) & 5u));
            }
#pragma unroll 1
            for (int q = kPB / 32 - 1; q >= 0; --q) {
                uint32_t bits = q == 0 ? hw[0] : q == 1 ? hw[1] : q == 2 ? hw[2] : hw[3];
                const int room = limit - q * 32;
                if (room <= 0) continue;
                if (room < 32) bits &= (1u << room) - 1u;
#pragma unroll 1
                for (; bits;) {
                    const int jj = 31 - __clz(bits);
                    bits &= ~(1u << jj);
                    const int j = q * 32 + jj;
                    const int pos = lo + j;
                    const Rec r = load_rec(P.rec[st][j]);
                    Eval e[2];
                    bool act[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) act[h] = pos < last[h] && eval_alpha<LP>(r, lx, ly[h], e[h]);
                    const uint32_t amask = __ballot_sync(0xffffffffu, act[0] || act[1]);
                    if (!amask) continue;
                    const uint32_t rid = P.val[st][j];
                    const int sid = static_cast<int>(static_cast<int64_t>(rid) - surf0);
                    const float4 col = P.rec[st][j][3];
                    float vals[kSlots];
#pragma unroll
                    for (int k2 = 0; k2 < kSlots; ++k2) vals[k2] = 0.0f;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (!act[h]) continue;
                        const float one_m = __fsub_rn(1.0f, e[h].alpha);
                        const float inv = rcp_approx(one_m); // one_m >= 0.01
                        const float Tj = Tc[h] * inv;
                        const float w = e[h].alpha * Tj;
                        const float dot = sel[h].match(a, pix[h], K, fp.n, sid);
                        const float sj = gr[h] * col.y + gg[h] * col.z + gb[h] * col.w + dot;
                        const float dLda = Tj * sj - suffix[h] * inv;
                        suffix[h] = fmaf(w, sj, suffix[h]);
                        Tc[h] = Tj;
                        vals[0] += w * gr[h];
                        vals[1] += w * gg[h];
                        vals[2] += w * gb[h];
                        if (LP && !e[h].clamped && e[h].filt) {
                            // rho = 2 |x - p0|^2: dL/dp0 = (-a / 2)(-4 (x - p0))
                            const float aa = dLda * e[h].alpha;
                            vals[3] += dLda * e[h].G;
                            vals[kSlots > 12 ? 11 : 0] += 2.0f * aa * e[h].dx;
                            vals[kSlots > 12 ? 12 : 0] += 2.0f * aa * e[h].dy;
                        } else if (!e[h].clamped) {
                            const float rq = rcp_approx(e[h].q2);
                            const float u = e[h].q0 * rq, vv = e[h].q1 * rq;
                            const float d2 = u * u + vv * vv;
                            const float aa = dLda * e[h].alpha;
                            vals[3] += dLda * e[h].G;
                            vals[4] += aa * u * u;
                            vals[5] += aa * u * vv;
                            vals[6] += aa * vv * vv;
                            vals[7] += aa * u;
                            vals[8] += aa * vv;
                            vals[9] += aa * d2 * u;
                            vals[10] += aa * d2 * vv;
                        }
                    }
                    add_record_sums<LP>(vals, act[0] || act[1], amask, lane,
                                        a.moments + static_cast<int64_t>(rid) * kM);
                }
            }
        }
        pipe_release(P, b);
    }
}

template <bool LP, int OCC, int TH = 16>
__global__ void __launch_bounds__(pair_threads(TH), OCC)
    render_bwd_pair_kernel(const __grid_constant__ FrameParams fp, BwdArgs a)
{
    __shared__ __align__(128) Pipe P;
    __shared__ int s_maxlast;
    __shared__ uint32_t s_next;
    uint32_t i = blockIdx.x;
    while (true) {
        const uint32_t tile = a.ranges[2 * fp.n_tiles_total + i];
        if (PSI_CHECK(tile < fp.n_tiles_total, kChkTile, a.status)) bwd_tile_pair<LP, TH>(fp, a, P, s_maxlast, tile);
        if (!a.work) break;
        __syncthreads();
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

// OCC: CTAs per SM the kernel is built for (the launch shape the autotuner
// picks). Tiles longest list first; the persistent launch (a.work set) fetches
// further tiles from the context's counter as the forward kernel does.
template <int KMAX, int DT, int CH, bool SAVED, bool LP, int OCC, int TH = 16, bool NW = false>
__global__ void __launch_bounds__(pipe_threads(TH), OCC)
    render_bwd_kernel(const __grid_constant__ FrameParams fp, BwdArgs a)
{
    __shared__ __align__(128) Pipe P;
    __shared__ int s_maxlast;
    __shared__ uint32_t s_next;
    uint32_t i = blockIdx.x;
    while (true) {
        const uint32_t tile = a.ranges[2 * fp.n_tiles_total + i];
        if (PSI_CHECK(tile < fp.n_tiles_total, kChkTile, a.status))
            bwd_tile<KMAX, DT, CH, SAVED, LP, TH, NW>(fp, a, P, s_maxlast, tile);
        if (!a.work) break;
        __syncthreads();
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

// Per record: dL/dM = T^T M'^-T W (M' = T M is the map shifted to the projected
// centre), then through M = [K R s_u t_u | K R s_v t_v | K (R mu + t)].
template <bool LP>
__global__ void __launch_bounds__(256) chain_kernel(const __grid_constant__ FrameParams fp, psi_surfels s,
                                                    const float4 *__restrict__ moments, psi_grads g)
{
    const int64_t total = fp.n * fp.n_views;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= total) return;
    constexpr int kV = moments_per_record(LP) / 4;
    // slots: dL/dc (3), dL/do, Suu, Suv, Svv, Su, Sv, Sdu, Sdv, pad[, dL/dp0 (2), pad (3)]
    const float4 q0 = moments[kV * r], q1 = moments[kV * r + 1], q2 = moments[kV * r + 2];
    const float2 gp = LP ? make_float2(moments[kV * r + 2].w, moments[kV * r + 3].x) : make_float2(0.0f, 0.0f);
    if (q0.x == 0.0f && q0.y == 0.0f && q0.z == 0.0f && q0.w == 0.0f && q1.x == 0.0f && q1.y == 0.0f &&
        q1.z == 0.0f && q1.w == 0.0f && q2.x == 0.0f && q2.y == 0.0f && q2.z == 0.0f && gp.x == 0.0f && gp.y == 0.0f)
        return;
    const int v = static_cast<int>(r / fp.n);
    const int64_t i = r - static_cast<int64_t>(v) * fp.n;
    const ViewParams &cam = fp.v[v];
    const float *R = cam.R;
    if (g.rgb) {
        if (q0.x != 0.0f) atomicAdd(g.rgb + 3 * i, q0.x);
        if (q0.y != 0.0f) atomicAdd(g.rgb + 3 * i + 1, q0.y);
        if (q0.z != 0.0f) atomicAdd(g.rgb + 3 * i + 2, q0.z);
    }
    if (g.opacity) atomicAdd(g.opacity + i, q0.w);
    const float Suu = q1.x, Suv = q1.y, Svv = q1.z, Su = q1.w, Sv = q2.x, Sdu = q2.y, Sdv = q2.z;

    float mu[3], tu[3], tv[3];
    for (int k = 0; k < 3; ++k) {
        mu[k] = s.mu[3 * i + k];
        tu[k] = s.tu[3 * i + k];
        tv[k] = s.tv[3 * i + k];
    }
    const float su = s.scale[2 * i], sv = s.scale[2 * i + 1];
    float xc[3], au[3], av[3];
    for (int k = 0; k < 3; ++k) {
        xc[k] = R[3 * k] * mu[0] + R[3 * k + 1] * mu[1] + R[3 * k + 2] * mu[2] + cam.t[k];
        au[k] = R[3 * k] * tu[0] + R[3 * k + 1] * tu[1] + R[3 * k + 2] * tu[2];
        av[k] = R[3 * k] * tv[0] + R[3 * k + 1] * tv[1] + R[3 * k + 2] * tv[2];
    }
    const float fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
    const float w = xc[2];
    const float p0x = (fx * xc[0] + cx * w) / w, p0y = (fy * xc[1] + cy * w) / w;
    // low-pass term: p0 = (fx X / Z + cx, fy Y / Z + cy), (X, Y, Z) = x_c
    float gxc[3] = {0.0f, 0.0f, 0.0f};
    if (LP) {
        gxc[0] = gp.x * fx / w;
        gxc[1] = gp.y * fy / w;
        gxc[2] = -(gp.x * fx * xc[0] + gp.y * fy * xc[1]) / (w * w);
    }
    // shifted columns of M'
    const float c0[3] = {fx * su * au[0] + (cx - p0x) * su * au[2], fy * su * au[1] + (cy - p0y) * su * au[2], su * au[2]};
    const float c1[3] = {fx * sv * av[0] + (cx - p0x) * sv * av[2], fy * sv * av[1] + (cy - p0y) * sv * av[2], sv * av[2]};
    const float c2[3] = {fx * xc[0] + (cx - p0x) * w, fy * xc[1] + (cy - p0y) * w, w};
    // rows of adj(M') (adj = det * M'^-1): c1 x c2, c2 x c0, c0 x c1
    float A[3][3];
    A[0][0] = c1[1] * c2[2] - c1[2] * c2[1];
    A[0][1] = c1[2] * c2[0] - c1[0] * c2[2];
    A[0][2] = c1[0] * c2[1] - c1[1] * c2[0];
    A[1][0] = c2[1] * c0[2] - c2[2] * c0[1];
    A[1][1] = c2[2] * c0[0] - c2[0] * c0[2];
    A[1][2] = c2[0] * c0[1] - c2[1] * c0[0];
    A[2][0] = c0[1] * c1[2] - c0[2] * c1[1];
    A[2][1] = c0[2] * c1[0] - c0[0] * c1[2];
    A[2][2] = c0[0] * c1[1] - c0[1] * c1[0];
    const float det = c0[0] * A[0][0] + c0[1] * A[0][1] + c0[2] * A[0][2];
    if (!(fabsf(det) > 0.0f)) {
        // a singular map: only the low-pass term has a gradient
        if (LP && g.mu)
            for (int k = 0; k < 3; ++k) atomicAdd(g.mu + 3 * i + k, R[k] * gxc[0] + R[3 + k] * gxc[1] + R[6 + k] * gxc[2]);
        return;
    }
    const float idet = 1.0f / det;
    const float W[3][3] = {{Suu, Suv, Su}, {Suv, Svv, Sv}, {-Sdu, -Sdv, -(Suu + Svv)}};
    // G' = M'^-T W = adj^T W / det
    float G[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = (A[0][a] * W[0][b] + A[1][a] * W[1][b] + A[2][a] * W[2][b]) * idet;
    // dL/dM = T^T G': third row picks up -p0x row0 - p0y row1
    for (int b = 0; b < 3; ++b) G[2][b] = G[2][b] - p0x * G[0][b] - p0y * G[1][b];
    // columns through K^T
    float guu[3], gvv[3];
    guu[0] = fx * G[0][0];
    guu[1] = fy * G[1][0];
    guu[2] = cx * G[0][0] + cy * G[1][0] + G[2][0];
    gvv[0] = fx * G[0][1];
    gvv[1] = fy * G[1][1];
    gvv[2] = cx * G[0][1] + cy * G[1][1] + G[2][1];
    gxc[0] += fx * G[0][2];
    gxc[1] += fy * G[1][2];
    gxc[2] += cx * G[0][2] + cy * G[1][2] + G[2][2];
    // uu = s_u R t_u, vv = s_v R t_v, xc = R mu + t
    float gsu = 0.0f, gsv = 0.0f;
    for (int k = 0; k < 3; ++k) {
        gsu += au[k] * guu[k];
        gsv += av[k] * gvv[k];
    }
    for (int k = 0; k < 3; ++k) {
        const float rtu = R[k] * guu[0] + R[3 + k] * guu[1] + R[6 + k] * guu[2];
        const float rtv = R[k] * gvv[0] + R[3 + k] * gvv[1] + R[6 + k] * gvv[2];
        const float rtx = R[k] * gxc[0] + R[3 + k] * gxc[1] + R[6 + k] * gxc[2];
        if (g.tu) atomicAdd(g.tu + 3 * i + k, su * rtu);
        if (g.tv) atomicAdd(g.tv + 3 * i + k, sv * rtv);
        if (g.mu) atomicAdd(g.mu + 3 * i + k, rtx);
    }
    if (g.scale) {
        atomicAdd(g.scale + 2 * i, gsu);
        atomicAdd(g.scale + 2 * i + 1, gsv);
    }
}

template <int KMAX, int CH, bool SAVED, bool LP, int OCC, int TH = 16>
cudaError_t launch_kcslo(const FrameParams &fp, const FeatView &f, const BwdArgs &a, cudaStream_t st)
{
    unsigned grid = fp.n_tiles_total;
    if (a.work) grid = persistent_grid(fp.n_tiles_total, OCC);
    constexpr int nt = pipe_threads(TH);
    if constexpr (KMAX == 0 && CH == 16) {
        // dense 16-channel tables: the register-held g_F row
        if (f.data && f.dim == 16) {
            switch (f.dtype) {
            case PSI_BF16: render_bwd_kernel<0, PSI_BF16, 16, SAVED, LP, OCC, TH, true><<<grid, nt, 0, st>>>(fp, a); break;
            case PSI_FP8_E4M3:
                render_bwd_kernel<0, PSI_FP8_E4M3, 16, SAVED, LP, OCC, TH, true><<<grid, nt, 0, st>>>(fp, a);
                break;
            default: render_bwd_kernel<0, PSI_F32, 16, SAVED, LP, OCC, TH, true><<<grid, nt, 0, st>>>(fp, a); break;
            }
            return cudaGetLastError();
        }
    }
    switch (f.data ? f.dtype : PSI_F32) {
    case PSI_BF16: render_bwd_kernel<KMAX, PSI_BF16, CH, SAVED, LP, OCC, TH><<<grid, nt, 0, st>>>(fp, a); break;
    case PSI_FP8_E4M3:
        render_bwd_kernel<KMAX, PSI_FP8_E4M3, CH, SAVED, LP, OCC, TH><<<grid, nt, 0, st>>>(fp, a);
        break;
    default: render_bwd_kernel<KMAX, PSI_F32, CH, SAVED, LP, OCC, TH><<<grid, nt, 0, st>>>(fp, a); break;
    }
    return cudaGetLastError();
}

// 16x8 tiles (Top-K with K <= 8, no low-pass filter): 4 pixel warps, 5 CTAs per SM
// (shared memory: one pipeline each)
constexpr int kOccTile8 = 5;

template <int KMAX, int CH, bool SAVED, bool LP>
cudaError_t launch_kcsl(const FrameParams &fp, const FeatView &f, const BwdArgs &a, bool alt, cudaStream_t st)
{
    // K <= 8: 3 CTAs per SM when pass A recomputes the Top-K set (the 4-CTA
    // build spills in the per-record reductions), 4 from saved state (56
    // registers, no Top-K in registers); larger K (register Top-K of 16 or
    // 32) and dense: 2 (the alternative shape: 4 resp. 3, and 1)
    constexpr bool small = KMAX > 0 && KMAX <= 8;
    constexpr int occ = small ? (SAVED ? 4 : 3) : 2;
    constexpr int occ_alt = small ? (SAVED ? 3 : 4) : 1;
    return alt ? launch_kcslo<KMAX, CH, SAVED, LP, occ_alt>(fp, f, a, st)
               : launch_kcslo<KMAX, CH, SAVED, LP, occ>(fp, f, a, st);
}

// Paired walk (saved state, Top-K): 4 pixel warps for a 16x16 tile, 2 for 16x8.
template <bool LP, int OCC, int TH>
cudaError_t launch_pair_o(const FrameParams &fp, const BwdArgs &a, cudaStream_t st)
{
    unsigned grid = fp.n_tiles_total;
    if (a.work) grid = persistent_grid(fp.n_tiles_total, OCC);
    render_bwd_pair_kernel<LP, OCC, TH><<<grid, pair_threads(TH), 0, st>>>(fp, a);
    return cudaGetLastError();
}

constexpr int kOccPair = 4, kOccPairAlt = 3, kOccPair8 = 5; // 43 KB of shared memory per CTA

cudaError_t launch_pair(const FrameParams &fp, const BwdArgs &a, bool alt, cudaStream_t st)
{
    if (fp.tile_h == 8) return launch_pair_o<false, kOccPair8, 8>(fp, a, st);
    if (fp.lowpass)
        return alt ? launch_pair_o<true, kOccPairAlt, 16>(fp, a, st) : launch_pair_o<true, kOccPair, 16>(fp, a, st);
    return alt ? launch_pair_o<false, kOccPairAlt, 16>(fp, a, st) : launch_pair_o<false, kOccPair, 16>(fp, a, st);
}

template <int KMAX, int CH, bool SAVED>
cudaError_t launch_kcs(const FrameParams &fp, const FeatView &f, const BwdArgs &a, bool alt, cudaStream_t st)
{
    return fp.lowpass ? launch_kcsl<KMAX, CH, SAVED, true>(fp, f, a, alt, st)
                      : launch_kcsl<KMAX, CH, SAVED, false>(fp, f, a, alt, st);
}

template <int KMAX, int CH>
cudaError_t launch_kc(const FrameParams &fp, const FeatView &f, const BwdArgs &a, bool alt, cudaStream_t st)
{
    return a.saved_T ? launch_kcs<KMAX, CH, true>(fp, f, a, alt, st) : launch_kcs<KMAX, CH, false>(fp, f, a, alt, st);
}

template <int KMAX>
cudaError_t launch_k(const FrameParams &fp, const FeatView &f, const BwdArgs &a, int ch, bool alt, cudaStream_t st)
{
    // the channel chunk only shapes the dense (K = 0) feature dot product
    if constexpr (KMAX > 0)
        return launch_kc<KMAX, 16>(fp, f, a, alt, st);
    else
        return ch == 32 ? launch_kc<KMAX, 32>(fp, f, a, alt, st) : launch_kc<KMAX, 16>(fp, f, a, alt, st);
}

} // namespace

namespace {
size_t moments_bytes(int64_t n_records, bool lp)
{
    return align_up(static_cast<size_t>(std::max<int64_t>(n_records, 1)) * moments_per_record(lp) * sizeof(float), 256);
}
} // namespace

// sized for the low-pass layout, which is the larger one
size_t render_bwd_workspace_bytes(int64_t n_records, int64_t n_pix, int top_k)
{
    const size_t kd = top_k > 0 ? align_up(static_cast<size_t>(n_pix) * top_k * sizeof(float), 256) : 0;
    return moments_bytes(n_records, true) + kd;
}

cudaError_t launch_render_bwd(const FrameParams &fp, const psi_surfels &s, const FeatView &f, const float4 *records,
                              const uint32_t *vals, const uint32_t *ranges, const float *g_rgb, const float *g_F,
                              const float *g_T, const psi_fwd_out *saved, const psi_grads &g, void *ws,
                              DevStatus *status, cudaStream_t st, cudaEvent_t const (*time_ev)[2], int shape)
{
    // optional timing events around one kernel (see psi_ctx_time_kernel)
    auto mark = [&](int kernel, int which) {
        if (time_ev && time_ev[kernel][which]) cudaEventRecord(time_ev[kernel][which], st);
    };
    const int64_t R = fp.n * fp.n_views;
    const bool lp = fp.lowpass != 0;
    cudaError_t e = cudaMemsetAsync(ws, 0, moments_bytes(R, lp), st);
    if (e != cudaSuccess || R == 0 || fp.n_tiles_total == 0) return e;
    BwdArgs a{};
    a.records = records;
    a.vals = vals;
    a.ranges = ranges;
    a.feat = f.data;
    a.wide = f.data && feat_rows_wide(f.data, f.dim, f.dtype);
    a.fscale = f.scale;
    a.D = f.dim;
    a.g_rgb = g_rgb;
    a.g_F = f.data ? g_F : nullptr;
    a.g_T = g_T;
    a.g_feat = f.data ? g.feat : nullptr;
    a.moments = static_cast<float *>(ws);
    a.status = status;
    if (saved) {
        a.saved_T = saved->T;
        a.saved_last = saved->n_last;
        a.saved_topk = saved->topk_ids;
        if (fp.top_k > 0 && a.g_F) {
            // feature terms from the saved selection: kd for the walk, dL/df
            float *kd = reinterpret_cast<float *>(static_cast<char *>(ws) + moments_bytes(R, lp));
            mark(PSI_KERNEL_BWD_FEAT, 0);
            e = launch_feat_bwd(fp, f, saved->topk_ids, saved->topk_w, a.g_F, kd, a.g_feat, status, st);
            if (e != cudaSuccess) return e;
            mark(PSI_KERNEL_BWD_FEAT, 1);
            a.kd_saved = kd;
        }
    }
    const int K = fp.top_k;
    const int ch = render_channel_chunk(f.dim, K, shape);
    const bool alt = shape & kShapeAltOcc;
    a.work = (shape & kShapePersistent) ? status->work + 2 : nullptr;
    mark(PSI_KERNEL_BWD_WALK, 0);
    if (a.saved_T && K > 0 && (shape & kShapePairWalk))
        e = launch_pair(fp, a, alt, st);
    else if (fp.tile_h == 8)
        e = a.saved_T ? launch_kcslo<8, 16, true, false, kOccTile8, 8>(fp, f, a, st)
                      : launch_kcslo<8, 16, false, false, kOccTile8, 8>(fp, f, a, st);
    else if (K == 0)
        e = launch_k<0>(fp, f, a, ch, alt, st);
    else if (K <= 8)
        e = launch_k<8>(fp, f, a, ch, alt, st);
    else if (K <= 16)
        e = launch_k<16>(fp, f, a, ch, alt, st);
    else
        e = launch_k<32>(fp, f, a, ch, alt, st);
    if (e != cudaSuccess) return e;
    mark(PSI_KERNEL_BWD_WALK, 1);
    if (lp)
        chain_kernel<true><<<static_cast<unsigned>((R + 255) / 256), 256, 0, st>>>(fp, s, static_cast<const float4 *>(ws), g);
    else
        chain_kernel<false><<<static_cast<unsigned>((R + 255) / 256), 256, 0, st>>>(fp, s, static_cast<const float4 *>(ws), g);
    return cudaGetLastError();
}

} // namespace psi
