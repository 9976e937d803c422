// Per-pixel surfel evaluation shared by the forward (a4) and adjoint (a5)
// compositing kernels, and the TMA staging of tile-list batches.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace psi {
namespace raster {

constexpr int kTile = 16;    // tile width in pixels (16x16 or 16x8 tiles), one thread per pixel
constexpr int kRecF4 = 5;    // render record: 80 bytes = 5 float4
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kNegHalfLog2e = -0.72134752044448170f; // -log2(e)/2: exp(-d2/2) = 2^(d2 * k)

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Thread -> pixel inside the 16x16 tile: warp w owns the 8x4 block at
// ((w & 1) * 8, (w >> 1) * 4); lane l is pixel (l & 7, l >> 3) of the block.
__device__ __forceinline__ void pixel_of_thread(int tid, int &lx, int &ly)
{
    const int w = tid >> 5, l = tid & 31;
    lx = (w & 1) * 8 + (l & 7);
    ly = (w >> 1) * 4 + (l >> 3);
}

// Staged render record after the per-tile transform: q = A (lx, ly, 1) with
// (lx, ly) the pixel's integer offset inside the tile; (ox, oy) = centre of the
// tile's first pixel minus the projected centre (the low-pass term's offset).
struct Rec {
    float a00, a01, c0, a10, a11, c1, a20, a21, c2;
    float o, r2;
    float ox, oy;
};

__device__ __forceinline__ Rec load_rec(const float4 *r)
{
    const float4 x = r[0], y = r[1], z = r[2], w = r[3];
    Rec q;
    q.a00 = x.x; q.a01 = x.y; q.c0 = x.z; q.a10 = x.w;
    q.a11 = y.x; q.c1 = y.y; q.a20 = y.z; q.a21 = y.w;
    q.c2 = z.x; q.o = z.w; q.r2 = w.x;
    q.ox = z.y; q.oy = z.z;
    return q;
}

struct Eval {
    float q0, q1, q2, d2, G, alpha;
    bool clamped;
    bool filt;    // low-pass filter only: its screen-space term won
    float dx, dy; // low-pass filter only: pixel centre minus projected centre
};

// alpha = min(0.99, o exp(-(u^2+v^2)/2)) of one surfel at one pixel (Sec. 3.1),
// (u, v) = (q0/q2, q1/q2). Returns false if the pixel lies outside the support
// disc (u^2+v^2 > r^2) or alpha < 1/255. Every operation is an explicitly
// rounded intrinsic, so forward and adjoint kernels reproduce the same alpha
// (and hence the same Top-K sets) bit for bit.
// LP: the 2DGS object-space low-pass filter. The Gaussian's argument is
// min(u^2+v^2, 2 (dx^2+dy^2)), (dx, dy) the pixel centre minus the projected
// centre (a screen-space Gaussian of standard deviation sqrt(2)/2 pixel), and
// the support is that argument <= r^2. The surfel's own term wins ties.
template <bool LP = false>
__device__ __forceinline__ bool eval_alpha(const Rec &r, float lx, float ly, Eval &e)
{
    e.q0 = __fmaf_rn(r.a00, lx, __fmaf_rn(r.a01, ly, r.c0));
    e.q1 = __fmaf_rn(r.a10, lx, __fmaf_rn(r.a11, ly, r.c1));
    e.q2 = __fmaf_rn(r.a20, lx, __fmaf_rn(r.a21, ly, r.c2));
    const float nn = __fmaf_rn(e.q0, e.q0, __fmul_rn(e.q1, e.q1));
    const float dd = __fmul_rn(e.q2, e.q2);
    if constexpr (LP) {
        const bool ell = (nn <= __fmul_rn(r.r2, dd)) && (dd > 0.0f);
        const float rho3 = ell ? __fmul_rn(nn, rcp_approx(dd)) : __int_as_float(0x7f800000);
        e.dx = __fadd_rn(lx, r.ox);
        e.dy = __fadd_rn(ly, r.oy);
        const float rho2 = __fmul_rn(2.0f, __fmaf_rn(e.dx, e.dx, __fmul_rn(e.dy, e.dy)));
        e.filt = rho2 < rho3;
        if (e.filt ? !(rho2 <= r.r2) : !ell) return false;
        e.d2 = e.filt ? rho2 : rho3;
    } else {
        if (!(nn <= __fmul_rn(r.r2, dd)) || !(dd > 0.0f)) return false;
        e.d2 = __fmul_rn(nn, rcp_approx(dd));
    }
    e.G = ex2_approx(__fmul_rn(e.d2, kNegHalfLog2e));
    const float a = __fmul_rn(r.o, e.G);
    e.clamped = a > kAlphaMax;
    e.alpha = e.clamped ? kAlphaMax : a;
    return e.alpha >= kAlphaMin;
}

// ------------------------------------------------------------ Top-K
// The K largest weights of one pixel with their list positions (Sec. 5, Top-K
// Hard Selection), kept sorted by weight (descending; among equal weights the
// earlier list position first), so the worst kept weight is always the last
// slot. A new weight enters only if it is strictly larger than that worst one
// -- it comes later in the list than everything kept, so ties favour the
// earlier surfel -- by one compare-and-shift pass. With a runtime K below
// KMAX the first KMAX-K slots hold +inf and never move. The insertion runs
// under a warp vote, so lanes pay one compare per surfel unless some lane of
// the warp improves its set.
template <int KMAX>
struct TopK {
    float w[KMAX];
    int p[KMAX];

    __device__ __forceinline__ void init(int K)
    {
#pragma unroll
        for (int s = 0; s < KMAX; ++s) {
            w[s] = (s < KMAX - K) ? __int_as_float(0x7f800000) : -1.0f;
            p[s] = 0x7fffffff;
        }
    }

    __device__ __forceinline__ void offer(bool hit, float wt, int pos)
    {
        const bool better = hit && wt > w[KMAX - 1];
        if (__any_sync(0xffffffffu, better)) {
            if (better) {
                bool gt[KMAX];
#pragma unroll
                for (int s = 0; s < KMAX; ++s) gt[s] = wt > w[s];
#pragma unroll
                for (int s = KMAX - 1; s > 0; --s) {
                    w[s] = gt[s - 1] ? w[s - 1] : (gt[s] ? wt : w[s]);
                    p[s] = gt[s - 1] ? p[s - 1] : (gt[s] ? pos : p[s]);
                }
                w[0] = gt[0] ? wt : w[0];
                p[0] = gt[0] ? pos : p[0];
            }
        }
    }

    // order the slots by list position (empty slots last)
    __device__ __forceinline__ void sort_by_pos()
    {
#pragma unroll
        for (int round = 0; round < KMAX; ++round) {
#pragma unroll
            for (int s = (round & 1); s + 1 < KMAX; s += 2) {
                if (p[s] > p[s + 1]) {
                    const int tp = p[s];
                    p[s] = p[s + 1];
                    p[s + 1] = tp;
                    const float tw = w[s];
                    w[s] = w[s + 1];
                    w[s + 1] = tw;
                }
            }
        }
    }

    __device__ __forceinline__ bool valid(int s, int K) const { return s < K && p[s] != 0x7fffffff; }
};

// ------------------------------------------------------------ decoupled pipeline
// A tile's list is streamed through kPS shared-memory stages of kPB records. A
// dedicated producer warp (the last warp) fills a stage with one TMA bulk copy
// per record (completion on full[s]), transforms the records for the tile once
// (ready[s]), and refills the stage after all pixel warps (8 for a 16x16 tile,
// 4 for 16x8) released it (empty[s], one arrival per pixel warp). Pixel warps only wait for ready stages, so a warp
// with little work in a batch runs ahead instead of waiting at a CTA barrier.
// Every wait is bounded; `alive` counts pixel warps with pixels still
// compositing (the producer stops when it reaches zero).
constexpr int kPS = 4;            // stages
constexpr int kPB = 128;          // records per stage (four 32-bit hit words per warp)
// pixel warps of a 16 x TH tile (8x4-pixel blocks, two per block row) and the
// CTA size with the producer warp
__host__ __device__ constexpr int pixel_warps(int TH) { return TH / 2; }
__host__ __device__ constexpr int pipe_threads(int TH) { return 32 * (pixel_warps(TH) + 1); }
constexpr int kPixelWarps = pixel_warps(16);
constexpr int kPipeThreads = pipe_threads(16);

struct Pipe {
    float4 rec[kPS][kPB][kRecF4];
    uint32_t val[kPS][kPB];
    uint64_t full[kPS], ready[kPS], empty[kPS];
    int alive;
    int abort;
};

__device__ __forceinline__ int vload(const int &x) { return *reinterpret_cast<const volatile int *>(&x); }

// thread 0; the caller synchronises the CTA afterwards. alive = the number of
// pixel warps (each releases every stage once per batch)
__device__ __forceinline__ void pipe_init(Pipe &P, int alive)
{
    for (int s = 0; s < kPS; ++s) {
        mbar_init(&P.full[s], 1);
        mbar_init(&P.ready[s], 1);
        mbar_init(&P.empty[s], alive);
    }
    P.alive = alive;
    P.abort = 0;
    fence_mbar_init();
}

// thread 0, between two tiles of a persistent CTA (after a CTA barrier):
// retire the barriers so that pipe_init may initialise them again
__device__ __forceinline__ void pipe_inval(Pipe &P)
{
    for (int s = 0; s < kPS; ++s) {
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&P.full[s])) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&P.ready[s])) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&P.empty[s])) : "memory");
    }
}

// Grid of a persistent compositing launch: occ CTAs per SM, at most one per tile.
inline unsigned persistent_grid(uint32_t n_tiles, int occ)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return static_cast<unsigned>(std::min<int64_t>(n_tiles, static_cast<int64_t>(occ) * sms));
}

// Batch b of a walk over n list entries (forward: from the front; reverse:
// from the back); returns the first list position and sets the count.
__device__ __forceinline__ int batch_range(int b, int n, bool reverse, int &cnt)
{
    const int nb = (n + kPB - 1) / kPB;
    const int bi = reverse ? nb - 1 - b : b;
    cnt = min(kPB, n - bi * kPB);
    return bi * kPB;
}

// Per-tile transform of one staged record: fold the tile origin into the
// third column so that q = A (lx, ly, 1) with small, exact pixel offsets, and
// replace the covered-pixel rectangle by the mask of the 8x4 warp blocks it
// meets (bit w = warp w), so a warp skips a record with one shared load.
__device__ __forceinline__ void transform_record(float4 *r, int tile_x0, int tile_y0)
{
    const float4 q = r[4];
    const uint32_t bx = __float_as_uint(q.x), by = __float_as_uint(q.y);
    const int x0 = static_cast<int>(bx & 0xFFFFu) - tile_x0, x1 = static_cast<int>(bx >> 16) - tile_x0;
    const int y0 = static_cast<int>(by & 0xFFFFu) - tile_y0, y1 = static_cast<int>(by >> 16) - tile_y0;
    uint32_t mask = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int cx = (w & 1) * 8, cy = (w >> 1) * 4;
        if (x0 <= cx + 7 && x1 >= cx && y0 <= cy + 3 && y1 >= cy) mask |= 1u << w;
    }
    r[4] = make_float4(q.x, q.y, __uint_as_float(mask), 0.0f);
    float4 x = r[0], y = r[1], z = r[2];
    const float ox = (static_cast<float>(tile_x0) + 0.5f) - z.y;
    const float oy = (static_cast<float>(tile_y0) + 0.5f) - z.z;
    x.z = __fmaf_rn(x.x, ox, __fmaf_rn(x.y, oy, x.z));
    y.y = __fmaf_rn(x.w, ox, __fmaf_rn(y.x, oy, y.y));
    z.x = __fmaf_rn(y.z, ox, __fmaf_rn(y.w, oy, z.x));
    z.y = ox; // the projected centre becomes the tile-relative offset (low-pass term)
    z.z = oy;
    r[0] = x;
    r[1] = y;
    r[2] = z;
}

// Producer warp: walks batches 0..nb-1 of the list (entries [list0, list0+n)),
// forward or reverse, until all batches are transformed or no pixel warp is
// alive. Returns false on a timeout (status raised, abort set).
__device__ __forceinline__ bool pipe_produce(Pipe &P, const uint32_t *__restrict__ vals, int64_t list0, int n,
                                             bool reverse, const float4 *__restrict__ records, int tile_x0,
                                             int tile_y0, DevStatus *st, int site, uint32_t rec_lo = 0,
                                             uint32_t rec_hi = 0xffffffffu)
{
    (void)rec_lo;
    (void)rec_hi;
    const int lane = threadIdx.x & 31;
    const int nb = (n + kPB - 1) / kPB;
    int issued = 0, done = 0; // batches issued / transformed
    unsigned long long t_idle = 0;
    const unsigned long long limit = wait_limit(st);
    bool ok = true;
    while (done < nb) {
        if (vload(P.alive) == 0 || vload(P.abort)) break;
        bool progressed = false;
        // transform the oldest issued batch once its copies have landed
        if (done < issued) {
            const int s = done % kPS;
            const bool landed = __shfl_sync(0xffffffffu, lane == 0 ? mbar_try_wait(&P.full[s], (done / kPS) & 1) : false, 0);
            if (landed) {
                int cnt;
                batch_range(done, n, reverse, cnt);
                for (int j = lane; j < cnt; j += 32) transform_record(P.rec[s][j], tile_x0, tile_y0);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&P.ready[s]);
                ++done;
                progressed = true;
            }
        }
        // issue the next batch into a stage every pixel warp has released
        if (issued < nb && issued < done + kPS) {
            const int s = issued % kPS;
            const bool free_ = issued < kPS ||
                               __shfl_sync(0xffffffffu, lane == 0 ? mbar_try_wait(&P.empty[s], ((issued / kPS) - 1) & 1) : false, 0);
            if (free_) {
                int cnt;
                const int lo = batch_range(issued, n, reverse, cnt);
                for (int j = lane; j < cnt; j += 32) {
                    uint32_t r = vals[list0 + lo + j];
                    // debug builds: a list entry must be a record of this tile's view
                    if (!PSI_CHECK(r >= rec_lo && r < rec_hi, kChkRecord, st)) r = rec_lo;
                    P.val[s][j] = r;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive_expect_tx(&P.full[s], static_cast<uint32_t>(cnt) * (16u * kRecF4));
                __syncwarp();
                for (int j = lane; j < cnt; j += 32)
                    bulk_g2s(&P.rec[s][j][0], records + kRecF4 * static_cast<size_t>(P.val[s][j]), 16u * kRecF4, &P.full[s]);
                ++issued;
                progressed = true;
            }
        }
        if (progressed) {
            t_idle = 0;
        } else {
            const unsigned long long now = global_ns();
            if (t_idle == 0) {
                t_idle = now;
            } else if (now - t_idle > limit) {
                if (lane == 0 && st) {
                    atomicCAS(&st->wait_site, 0, site);
                    raise_status(st, PSI_ERR_TIMEOUT);
                    atomicExch(&P.abort, 1);
                }
                ok = false;
                break;
            }
            __nanosleep(64);
        }
    }
    // copies still in flight must land before the stages are reused or freed
    for (int b = done; b < issued; ++b) {
        if (lane == 0) mbar_wait(&P.full[b % kPS], (b / kPS) & 1, st, kSiteDrain);
        __syncwarp();
    }
    return ok;
}

// Pixel warp (all 32 lanes): wait until batch b is ready. Returns false if
// the walk is over for everyone (no pixel warp alive, or an abort). The
// answer is the same in every lane of the warp: once one lane has seen the
// batch ready it stays ready (the stage cannot be refilled before this warp
// releases it), so the others wait for it too.
__device__ __forceinline__ bool pipe_wait_ready(Pipe &P, int b, DevStatus *st, int site)
{
    const int s = b % kPS;
    const uint32_t par = (b / kPS) & 1;
    bool ready = mbar_try_wait(&P.ready[s], par);
    if (!ready) {
        const unsigned long long limit = wait_limit(st);
        const unsigned long long t0 = global_ns();
        while (true) {
            if (mbar_try_wait(&P.ready[s], par)) {
                ready = true;
                break;
            }
            if (vload(P.abort) || vload(P.alive) == 0) break;
            if (global_ns() - t0 > limit) {
                if (st) {
                    atomicCAS(&st->wait_site, 0, site);
                    raise_status(st, PSI_ERR_TIMEOUT);
                }
                atomicExch(&P.abort, 1);
                break;
            }
        }
    }
    if (!__any_sync(0xffffffffu, ready)) return false;
    if (!ready) mbar_wait(&P.ready[s], par, st, site); // complete already: returns at once
    return true;
}

// Pixel warp: done with batch b (one arrival per warp).
__device__ __forceinline__ void pipe_release(Pipe &P, int b)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&P.empty[b % kPS]);
}

__device__ __forceinline__ bool pipe_hits(const Pipe &P, int s, int j, int w)
{
    return (__float_as_uint(P.rec[s][j][4].z) >> w) & 1u;
}

// Bitmap of the records of stage s (cnt of them) that touch warp w's block:
// bit (j & 31) of word j >> 5. Identical in every lane.
__device__ __forceinline__ void pipe_hit_words(const Pipe &P, int s, int cnt, int w, uint32_t hw[kPB / 32])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < kPB / 32; ++q) {
        const int j = q * 32 + lane;
        hw[q] = __ballot_sync(0xffffffffu, j < cnt && pipe_hits(P, s, j, w));
    }
}

// ------------------------------------------------------------ features
// 32 bytes of read-only global memory (address 32-byte aligned).
__device__ __forceinline__ void ldg32(const void *p, uint32_t w[8])
{
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
        : "l"(p));
}

// Whether feature rows can be read 32 bytes at a time: the table starts on a
// 32-byte boundary and every row is a whole number of 32-byte units.
inline bool feat_rows_wide(const void *base, int D, int dtype)
{
    const int esize = dtype == PSI_F32 ? 4 : (dtype == PSI_BF16 ? 2 : 1);
    return (reinterpret_cast<uintptr_t>(base) % 32 == 0) && ((D * esize) % 32 == 0);
}

// CH (16 or 32) channels [c0, c0+CH) of feature row i as float32, before the
// per-channel scale. Rows are read with 16-byte vector loads, or 32-byte ones
// when `wide` (see feat_rows_wide; c0 is a multiple of 16): a lane then
// touches one whole 32-byte sector per load when the rows of a warp differ.
template <int DT, int CH>
__device__ __forceinline__ void load_feat(const void *__restrict__ base, int64_t i, int D, int c0, float *f,
                                          bool wide = false)
{
    if (wide && DT != PSI_FP8_E4M3) {
        const unsigned char *row = static_cast<const unsigned char *>(base) + (i * D + c0) * (DT == PSI_F32 ? 4 : 2);
        if constexpr (DT == PSI_F32) {
#pragma unroll
            for (int k = 0; k < CH / 8; ++k) {
                uint32_t w[8];
                ldg32(row + 32 * k, w);
#pragma unroll
                for (int h = 0; h < 8; ++h) f[8 * k + h] = __uint_as_float(w[h]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < CH / 16; ++k) {
                uint32_t w[8];
                ldg32(row + 32 * k, w);
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    f[16 * k + 2 * h] = __uint_as_float(w[h] << 16);
                    f[16 * k + 2 * h + 1] = __uint_as_float(w[h] & 0xFFFF0000u);
                }
            }
        }
        return;
    }
    if constexpr (DT == PSI_F32) {
        const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(base) + i * D + c0);
#pragma unroll
        for (int k = 0; k < CH / 4; ++k) {
            const float4 v = __ldg(p + k);
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
    } else if constexpr (DT == PSI_BF16) {
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(base) + i * D + c0);
#pragma unroll
        for (int k = 0; k < CH / 8; ++k) {
            const uint4 v = __ldg(p + k);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                f[8 * k + 2 * h] = __uint_as_float(w[h] << 16);
                f[8 * k + 2 * h + 1] = __uint_as_float(w[h] & 0xFFFF0000u);
            }
        }
    } else {
        // FP8 E4M3 (sign, 4 exponent bits with bias 7, 3 mantissa bits): placing
        // the 7 magnitude bits at float bits [20, 27) gives 2^(e-127)(1+m/8)
        // (or the denormal m 2^-129 when e = 0); times 2^120 that is exactly
        // 2^(e-7)(1+m/8) (or m 2^-9).
        const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const uint8_t *>(base) + i * D + c0);
#pragma unroll
        for (int k = 0; k < CH / 16; ++k) {
            const uint4 v = __ldg(p + k);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t byte = (w[h] >> (8 * b)) & 0xFFu;
                    const uint32_t bits = ((byte & 0x80u) << 24) | ((byte & 0x7Fu) << 20);
                    f[16 * k + 4 * h + b] = __uint_as_float(bits) * 0x1p120f;
                }
            }
        }
    }
}

// Four channels [c, c + 4) of feature row i as float32 (before the scale).
template <int DT>
__device__ __forceinline__ float4 load_feat4(const void *__restrict__ base, int64_t i, int D, int c)
{
    if constexpr (DT == PSI_F32) {
        return __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + i * D + c));
    } else if constexpr (DT == PSI_BF16) {
        const uint2 u = __ldg(reinterpret_cast<const uint2 *>(static_cast<const __nv_bfloat16 *>(base) + i * D + c));
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u), __uint_as_float(u.y << 16),
                           __uint_as_float(u.y & 0xFFFF0000u));
    } else {
        // FP8 E4M3: the 7 magnitude bits at float bits [20, 27), times 2^120
        // (as in load_feat)
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(static_cast<const uint8_t *>(base) + i * D + c));
        float f[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t byte = (w >> (8 * b)) & 0xFFu;
            f[b] = __uint_as_float(((byte & 0x80u) << 24) | ((byte & 0x7Fu) << 20)) * 0x1p120f;
        }
        return make_float4(f[0], f[1], f[2], f[3]);
    }
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc)
{
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}

// Store CH channels (times scale) of one pixel's feature row as FP32 or BF16.
template <int CH>
__device__ __forceinline__ void store_feat(void *F, bool bf16, int64_t pix, int D, int c0, const float *acc,
                                           const float *__restrict__ scale)
{
    float v[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = scale ? acc[c] * __ldg(scale + c0 + c) : acc[c];
    if (bf16) {
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(F) + pix * D + c0);
#pragma unroll
        for (int k = 0; k < CH / 8; ++k) {
            uint32_t w4[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * k + 2 * h], v[8 * k + 2 * h + 1]);
                w4[h] = *reinterpret_cast<const uint32_t *>(&p2);
            }
            dst[k] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    } else {
        float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(F) + pix * D + c0);
#pragma unroll
        for (int k = 0; k < CH / 4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
}

// ------------------------------------------------------------ warp sums
// Sum 16 per-lane values over the warp (transposing butterfly, 16 shuffles):
// afterwards lane l (and l ^ 1) holds the total of value index
// 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of l).
__device__ __forceinline__ float warp_transpose_sum16(float v[16], int lane)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool hi = lane & 16;
        const float send = hi ? v[k] : v[k + 8];
        const float keep = hi ? v[k + 8] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool hi = lane & 8;
        const float send = hi ? v[k] : v[k + 4];
        const float keep = hi ? v[k + 4] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const bool hi = lane & 4;
        const float send = hi ? v[k] : v[k + 2];
        const float keep = hi ? v[k + 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        const float send = hi ? v[0] : v[1];
        const float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

} // namespace raster
} // namespace psi
