// Frustum-constrained cross-attention (Sec. 4.1) on the 5th-generation tensor
// cores, forward and adjoint.
//
// Over the surfels j whose 99 % confidence disc meets the view frustum (the
// disc's bounding sphere, radius sqrt(chi2_2(0.99)) max(s_u, s_v), against the
// near plane and the four side planes of the image rectangle):
//     K_j = f_j + psi(mu_j),  V_j = f_j
//     e_ij = (Q_i W_Q)(K_j W_K)^T / sqrt(d),  Q'_i = softmax_j(e_ij) (V_j W_V)
// psi: channel c encodes axis c mod 3 with sin (t = c / 3 even) or cos (t odd)
// at frequency 10000^(-6k/C), k = t / 2.
//
// By associativity the per-surfel projections fold into the queries:
//     e_ij = qh_i . K_j,  qh_i = (Q_i W_Q) W_K^T / sqrt(d)   [n_q x C]
//     Q'_i = O_i W_V,     O_i = sum_j P_ij V_j              [n_q x C]
// so the work that scales with the surfels is two contractions per tile of
// 128 surfels -- S = qh [f | psi]^T over the C channels and O += P f over the
// surfels -- on the tensor cores (BF16 operands, FP32 accumulation in TMEM),
// plus an online softmax; the feature table is read once. A persistent CTA
// per SM walks a contiguous range of tiles:
//   warp 0     TMA: the resident qh tile, then the feature tiles (2-stage ring)
//   warp 1     TMEM allocation; one thread issues the MMAs
//   warps 2, 3, 8, 9  per tile, one surfel per thread: the frustum mask and
//              the psi row (BF16, 2 stages), one sin/cos pair per (axis,
//              frequency)
//   warps 4-7  one query row per thread: online softmax of S (double-buffered
//              in TMEM), P written to shared memory as the A operand of the
//              P f product, the O accumulator rescaled in TMEM when the row
//              maximum grows
// The feature tile is the K-major B operand of S and, read as an MN-major
// operand, the B operand of P f. Each CTA leaves (max, sum, O) per query; a
// combine kernel merges them and applies W_V.
//
// The adjoint (L = <G, Q'>): dO_i = G_i W_V^T, D_i = dO_i . O_i (normalised O),
// and per tile, with P recomputed from the forward's per-query max and sum:
//     dP_ij = dO_i . f_j,  dE_ij = P_ij (dP_ij - D_i)
//     dqh  += dE [f | psi]            (over the surfels, in TMEM across tiles)
//     dK_j  = sum_i dE_ij qh_i,  dV_j = sum_i P_ij dO_i   (per surfel)
// then dL/df_j += dK_j + dV_j and dL/dmu_j += dK_j . dpsi/dmu (active surfels),
// and the small products to Q, W_Q, W_K, W_V.
#include <cuda_bf16.h>

#include "tc.cuh"

namespace psi {
namespace {

using namespace tc;

constexpr float kChi2_99 = 9.21034037198f; // -2 ln 0.01
constexpr float kLnB = 9.21034037198f;     // ln 10000
constexpr float kLog2e = 1.4426950408889634f;
constexpr int kAT = 128;         // surfels per tile
constexpr int kAThreads = 320;   // 10 warps: TMA, MMA, 4 softmax, 4 psi (warps 2, 3, 8, 9)
constexpr uint32_t kAtom = 128u * 128u; // bytes of one 128-row x 128-byte swizzle atom column

struct AttnCam {
    float R[9], t[3];
    float fx, fy, cx, cy, W, H, z_near;
};

// The frustum test: the 99 % disc's bounding sphere is not wholly behind the
// near plane or outside a side plane of the image rectangle.
__device__ __forceinline__ bool frustum_active(const AttnCam &a, float mx, float my, float mz, float su, float sv)
{
    const float x = a.R[0] * mx + a.R[1] * my + a.R[2] * mz + a.t[0];
    const float y = a.R[3] * mx + a.R[4] * my + a.R[5] * mz + a.t[1];
    const float z = a.R[6] * mx + a.R[7] * my + a.R[8] * mz + a.t[2];
    const float r = sqrtf(kChi2_99) * fmaxf(su, sv);
    float d = z - a.z_near;
    d = fminf(d, (a.fx * x + a.cx * z) * rsqrtf(a.fx * a.fx + a.cx * a.cx));
    d = fminf(d, (-a.fx * x + (a.W - a.cx) * z) * rsqrtf(a.fx * a.fx + (a.W - a.cx) * (a.W - a.cx)));
    d = fminf(d, (a.fy * y + a.cy * z) * rsqrtf(a.fy * a.fy + a.cy * a.cy));
    d = fminf(d, (-a.fy * y + (a.H - a.cy) * z) * rsqrtf(a.fy * a.fy + (a.H - a.cy) * (a.H - a.cy)));
    return d + r >= 0.0f;
}

// Byte offset of the 16-byte chunk `chunk` (0..C/8-1) of row `row` (0..127) in
// a [128 x C] BF16 tile stored as C/64 column atoms of 128-byte rows with the
// 128-byte swizzle (the layout TMA writes and the MMA descriptors read).
__device__ __forceinline__ uint32_t tile_off(int row, int chunk)
{
    return static_cast<uint32_t>(chunk >> 3) * kAtom + static_cast<uint32_t>(row) * 128u +
           (static_cast<uint32_t>((chunk & 7) ^ (row & 7)) << 4);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// psi row of one centre as a row of a swizzled BF16 tile: channels 6k..6k+5
// are sin(m_x w_k), sin(m_y w_k), sin(m_z w_k), cos(m_x w_k), cos(m_y w_k),
// cos(m_z w_k) (t = c / 3, axis = c mod 3, k = t / 2), one sin/cos pair per
// (axis, k); w: frequency per k
template <int C>
__device__ __forceinline__ void psi_row(uint32_t tile, int row, float mx, float my, float mz, const float *w)
{
    float v[C];
#pragma unroll
    for (int k = 0; 6 * k < C; ++k) {
        float sn[3], cs[3];
        __sincosf(mx * w[k], &sn[0], &cs[0]);
        __sincosf(my * w[k], &sn[1], &cs[1]);
        __sincosf(mz * w[k], &sn[2], &cs[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (6 * k + a < C) v[6 * k + a] = sn[a];
            if (6 * k + 3 + a < C) v[6 * k + 3 + a] = cs[a];
        }
    }
#pragma unroll
    for (int ch = 0; ch < C / 8; ++ch)
        st_shared_v4(tile + tile_off(row, ch), pack_bf16(v[8 * ch], v[8 * ch + 1]), pack_bf16(v[8 * ch + 2], v[8 * ch + 3]),
                     pack_bf16(v[8 * ch + 4], v[8 * ch + 5]), pack_bf16(v[8 * ch + 6], v[8 * ch + 7]));
}

// the transform warps (2, 3, 8, 9) -> index 0..3 (the 32-row group of the tile they handle)
__device__ __forceinline__ int psi_warp_index(int wid) { return wid < 4 ? wid - 2 : wid - 6; }
__device__ __forceinline__ bool is_psi_warp(int wid) { return wid == 2 || wid == 3 || wid == 8 || wid == 9; }

// Shared-memory matrix descriptor for an MN-major operand in the 128-byte
// swizzle layout: 64-element (128-byte) rows along MN, 8 rows along K per
// 1024-byte group; lbo = byte stride between 64-element MN atoms, sbo = byte
// stride between 8-row K groups.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Bounded wait of one thread on an mbarrier phase that also gives up when
// another role of the CTA has aborted.
__device__ __forceinline__ bool await(uint64_t *bar, uint32_t parity, DevStatus *st, int site, int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long limit = wait_limit(st);
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*reinterpret_cast<volatile int *>(abort_flag)) return false;
        if (global_ns() - t0 > limit) {
            if (st) {
                atomicCAS(&st->wait_site, 0, site);
                raise_status(st, PSI_ERR_TIMEOUT);
            }
            atomicExch(abort_flag, 1);
            return false;
        }
    }
}

// all lanes of a warp wait; the answer is made warp-uniform
__device__ __forceinline__ bool await_warp(uint64_t *bar, uint32_t parity, DevStatus *st, int site, int *abort_flag)
{
    return __all_sync(0xffffffffu, await(bar, parity, st, site, abort_flag));
}

struct AttnParams {
    int64_t n;
    int n_tiles;
    int n_q;
    const AttnCam *camd; // the view, written to the workspace by the forward
    const float *mu;
    const float *scale;
    // forward: per CTA partials m [G][128], l [G][128], O [G][128][C]
    float *part_m, *part_l, *part_o;
    // adjoint: per-query max (log2 units) and 1 / sum, D_i; dqh partials [G][128][C]
    const float *M, *Linv, *Dq;
    float *part_dq;
    float *g_feat, *g_mu;
    DevStatus *status;
};

// shared-memory plan (dynamic, 1024-aligned): see attn_smem_bytes
template <int C>
struct FwdSmem {
    static constexpr uint32_t TILE = (C / 64) * kAtom; // [128 x C] BF16 tile
    static constexpr uint32_t Q = 0;                    // qh
    static constexpr uint32_t F = Q + TILE;             // feature ring [2]
    static constexpr uint32_t PSI = F + 2 * TILE;       // psi ring [2]
    static constexpr uint32_t P = PSI + 2 * TILE;       // P [128 q x 128 j] BF16 (2 atoms)
    static constexpr uint32_t BYTES = P + 2 * kAtom;
};

template <int C>
__global__ void __launch_bounds__(kAThreads, 1)
    attn_fwd_kernel(const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_q, AttnParams p)
{
    using L = FwdSmem<C>;
    constexpr int A = C / 64;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sb = smem_u32(base);
    __shared__ uint64_t f_full[2], f_empty[2], psi_full[2], psi_empty[2], s_full[2], s_empty[2], m_full[4];
    __shared__ uint64_t o_full, p_full, q_bar, drain_bar;
    __shared__ uint32_t mask[4][4];
    __shared__ float wk[C / 6 + 2];
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    __shared__ AttnCam cam_s;

    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    if (tid < static_cast<int>(sizeof(AttnCam) / 4))
        reinterpret_cast<float *>(&cam_s)[tid] = reinterpret_cast<const float *>(p.camd)[tid];
    const int t0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * p.n_tiles / gridDim.x);
    const int t1 = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * p.n_tiles / gridDim.x);
    const int nt = t1 - t0;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&f_full[i], 1);
            mbar_init(&f_empty[i], 1);
            mbar_init(&psi_full[i], 4);
            mbar_init(&psi_empty[i], 1);
            mbar_init(&s_full[i], 1);
            mbar_init(&s_empty[i], 4);
        }
        for (int i = 0; i < 4; ++i) mbar_init(&m_full[i], 4);
        mbar_init(&o_full, 1);
        mbar_init(&p_full, 4);
        mbar_init(&q_bar, 1);
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    for (int k = tid; k < C / 6 + 2; k += kAThreads)
        wk[k] = expf(-kLnB * 6.0f * static_cast<float>(k) / static_cast<float>(C));
    if (wid == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    DevStatus *st = p.status;

    if (wid == 0) {
        // ---------------- TMA producer
        int issued = 0, landed_q = 0;
        if (lane == 0 && nt > 0) {
            mbar_arrive_expect_tx(&q_bar, L::TILE);
            for (int a = 0; a < A; ++a) tma_load_2d(base + L::Q + a * kAtom, &map_q, a * 64, 0, &q_bar);
            landed_q = 1;
            for (int t = 0; t < nt; ++t) {
                const int s = t & 1;
                if (t >= 2 && !await(&f_empty[s], ((t >> 1) - 1) & 1, st, kSiteDecodeLoad, &abort_flag)) break;
                mbar_arrive_expect_tx(&f_full[s], L::TILE);
                for (int a = 0; a < A; ++a)
                    tma_load_2d(base + L::F + s * L::TILE + a * kAtom, &map_f, a * 64, (t0 + t) * kAT, &f_full[s]);
                ++issued;
            }
            // every started copy lands before the CTA's shared memory is released
            if (landed_q) mbar_wait(&q_bar, 0, st, kSiteDrain);
            for (int t = (issued > 2 ? issued - 2 : 0); t < issued; ++t) mbar_wait(&f_full[t & 1], (t >> 1) & 1, st, kSiteDrain);
        }
    } else if (wid == 1) {
        // ---------------- MMA issuer
        if (lane == 0 && nt > 0) {
            const uint32_t idesc_s = idesc_bf16(128, kAT);
            const uint32_t idesc_o = idesc_bf16(128, C) | (1u << 16); // B (the feature tile) MN-major
            bool ok = await(&q_bar, 0, st, kSiteDecodeQ, &abort_flag);
            // issue whichever product is ready: S of the next tile (its feature
            // and psi tiles landed, its S buffer released) or P f of the oldest
            // tile whose weights are written; bounded by the wait limit of the
            // context while nothing is ready
            int s_next = 0, pv_next = 0;
            const unsigned long long limit = wait_limit(st);
            unsigned long long t_idle = 0;
            while (ok && pv_next < nt) {
                bool progressed = false;
                if (s_next < nt) {
                    const int t = s_next, b = t & 1;
                    if (mbar_try_wait(&f_full[b], (t >> 1) & 1) && mbar_try_wait(&psi_full[b], (t >> 1) & 1) &&
                        (t < 2 || mbar_try_wait(&s_empty[b], ((t >> 1) - 1) & 1))) {
                        tc_fence_after();
                        const uint32_t d = tmem + b * kAT;
#pragma unroll 1
                        for (int k = 0; k < C / 16; ++k) {
                            const uint32_t off = (k >> 2) * kAtom + (k & 3) * 32;
                            const uint64_t a = sw128_desc(sb + L::Q + off);
                            mma_bf16(d, a, sw128_desc(sb + L::F + b * L::TILE + off), idesc_s, k > 0 ? 1u : 0u);
                            mma_bf16(d, a, sw128_desc(sb + L::PSI + b * L::TILE + off), idesc_s, 1u);
                        }
                        mma_commit(&s_full[b]);
                        mma_commit(&psi_empty[b]);
                        ++s_next;
                        progressed = true;
                    }
                }
                if (pv_next < s_next && mbar_try_wait(&p_full, pv_next & 1)) {
                    const int u = pv_next;
                    tc_fence_after();
                    const uint32_t fs = sb + L::F + (u & 1) * L::TILE;
#pragma unroll 1
                    for (int k = 0; k < kAT / 16; ++k) {
                        const uint64_t a = sw128_desc(sb + L::P + (k >> 2) * kAtom + (k & 3) * 32);
                        const uint64_t b = sw128_desc_mn(fs + k * 2048, kAtom, 1024);
                        mma_bf16(tmem + 256, a, b, idesc_o, (u > 0 || k > 0) ? 1u : 0u);
                    }
                    mma_commit(&o_full);
                    mma_commit(&f_empty[u & 1]);
                    ++pv_next;
                    progressed = true;
                }
                if (progressed) {
                    t_idle = 0;
                } else if (*reinterpret_cast<volatile int *>(&abort_flag)) {
                    ok = false;
                } else {
                    const unsigned long long now = global_ns();
                    if (t_idle == 0) {
                        t_idle = now;
                    } else if (now - t_idle > limit) {
                        if (st) {
                            atomicCAS(&st->wait_site, 0, kSiteDecodeMma);
                            raise_status(st, PSI_ERR_TIMEOUT);
                        }
                        atomicExch(&abort_flag, 1);
                        ok = false;
                    }
                }
            }
            // let every issued MMA group complete before TMEM is released
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, st, kSiteDrain);
        }
    } else if (is_psi_warp(wid)) {
        // ---------------- frustum mask and psi tiles, one surfel per thread
        const int gq = psi_warp_index(wid), row = gq * 32 + lane;
        // this thread's centre and scales, loaded one tile ahead
        auto fetch = [&](int t, float *m5) {
            const int64_t j = static_cast<int64_t>(t0 + t) * kAT + row;
            const bool valid = t < nt && j < p.n;
            m5[0] = valid ? p.mu[3 * j] : 0.f;
            m5[1] = valid ? p.mu[3 * j + 1] : 0.f;
            m5[2] = valid ? p.mu[3 * j + 2] : 0.f;
            m5[3] = valid ? p.scale[2 * j] : -1.f;
            m5[4] = valid ? p.scale[2 * j + 1] : -1.f;
        };
        float nx[5];
        fetch(0, nx);
        for (int t = 0; t < nt; ++t) {
            const int b = t & 1;
            const float mx = nx[0], my = nx[1], mz = nx[2], su = nx[3], sv = nx[4];
            fetch(t + 1, nx);
            if (t >= 2 && !await_warp(&psi_empty[b], ((t >> 1) - 1) & 1, st, kSiteDecodeMma, &abort_flag)) break;
            const bool act = su >= 0.f && frustum_active(cam_s, mx, my, mz, su, sv);
            const uint32_t word = __ballot_sync(0xffffffffu, act);
            if (lane == 0) mask[t & 3][gq] = word;
            __syncwarp();
            if (lane == 0) mbar_arrive(&m_full[t & 3]);
            psi_row<C>(sb + L::PSI + b * L::TILE, row, mx, my, mz, wk);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&psi_full[b]);
        }
    } else {
        // ---------------- softmax: one query row per thread
        const int q4 = wid & 3;
        const int row = q4 * 32 + lane;
        const uint32_t lane_bits = static_cast<uint32_t>(q4 * 32) << 16;
        float m_run = -__int_as_float(0x7f800000), l_run = 0.0f;
        bool ok = true;
        for (int t = 0; t < nt && ok; ++t) {
            const int b = t & 1;
            ok = await_warp(&m_full[t & 3], (t >> 2) & 1, st, kSiteDecodeMma, &abort_flag) &&
                 await_warp(&s_full[b], (t >> 1) & 1, st, kSiteDecodeMma, &abort_flag);
            if (!ok) break;
            uint32_t mw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) mw[k] = mask[t & 3][k];
            tc_fence_after();
            // pass 1 over the row: the maximum of the active scores (log2 units)
            float mt = -__int_as_float(0x7f800000);
#pragma unroll 1
            for (int c0 = 0; c0 < kAT; c0 += 32) {
                uint32_t s[32];
                tmem_ld16_async(tmem + lane_bits + b * kAT + c0, s);
                tmem_ld16_async(tmem + lane_bits + b * kAT + c0 + 16, s + 16);
                tmem_wait_ld();
                const uint32_t mword = mw[c0 >> 5];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj)
                    if ((mword >> jj) & 1u) mt = fmaxf(mt, __uint_as_float(s[jj]) * kLog2e);
            }
            const float m_new = fmaxf(m_run, mt);
            // P f of the previous tile has landed: the P buffer is free, O may be rescaled
            if (t >= 1) {
                ok = await_warp(&o_full, (t - 1) & 1, st, kSiteDecodeMma, &abort_flag);
                if (!ok) break;
                tc_fence_after();
                if (__any_sync(0xffffffffu, m_new > m_run)) {
                    const float scale_o = (m_new > m_run) ? ex2f(m_run - m_new) : 1.0f;
#pragma unroll 1
                    for (int c0 = 0; c0 < C; c0 += 16) {
                        uint32_t o[16];
                        tmem_ld16_async(tmem + lane_bits + 256 + c0, o);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 16; ++e) o[e] = __float_as_uint(__uint_as_float(o[e]) * scale_o);
                        tmem_st16(tmem + lane_bits + 256 + c0, o);
                    }
                    tmem_wait_st();
                }
            }
            const float alpha = (m_new > m_run) ? ex2f(m_run - m_new) : 1.0f;
            const bool any = m_new > -__int_as_float(0x7f800000);
            // pass 2: the weights, rounded to BF16 as the A operand of P f
            float psum = 0.0f;
#pragma unroll 1
            for (int c0 = 0; c0 < kAT; c0 += 32) {
                uint32_t s[32];
                tmem_ld16_async(tmem + lane_bits + b * kAT + c0, s);
                tmem_ld16_async(tmem + lane_bits + b * kAT + c0 + 16, s + 16);
                tmem_wait_ld();
                const uint32_t mword = any ? mw[c0 >> 5] : 0u;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j0 = ch * 8 + 2 * e, j1 = j0 + 1;
                        const float p0 = ((mword >> j0) & 1u) ? ex2f(__uint_as_float(s[j0]) * kLog2e - m_new) : 0.0f;
                        const float p1 = ((mword >> j1) & 1u) ? ex2f(__uint_as_float(s[j1]) * kLog2e - m_new) : 0.0f;
                        w[e] = pack_bf16(p0, p1);
                        // the sum of the values the tensor cores see
                        psum += __uint_as_float(w[e] << 16) + __uint_as_float(w[e] & 0xFFFF0000u);
                    }
                    st_shared_v4(sb + L::P + tile_off(row, (c0 >> 3) + ch), w[0], w[1], w[2], w[3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[b]);
            l_run = l_run * alpha + psum;
            m_run = m_new;
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&p_full);
        }
        if (ok && nt > 0) ok = await_warp(&o_full, (nt - 1) & 1, st, kSiteDecodeMma, &abort_flag);
        if (ok && nt > 0) {
            tc_fence_after();
            float *dst = p.part_o + (static_cast<int64_t>(blockIdx.x) * 128 + row) * C;
#pragma unroll 1
            for (int c0 = 0; c0 < C; c0 += 16) {
                uint32_t o[16];
                tmem_ld16_async(tmem + lane_bits + 256 + c0, o);
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; e += 4)
                    *reinterpret_cast<float4 *>(dst + c0 + e) =
                        make_float4(__uint_as_float(o[e]), __uint_as_float(o[e + 1]), __uint_as_float(o[e + 2]),
                                    __uint_as_float(o[e + 3]));
            }
            p.part_m[blockIdx.x * 128 + row] = m_run;
            p.part_l[blockIdx.x * 128 + row] = l_run;
        } else {
            p.part_m[blockIdx.x * 128 + row] = -__int_as_float(0x7f800000);
            p.part_l[blockIdx.x * 128 + row] = 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

// ------------------------------------------------------------------ adjoint
// shared-memory plan of the adjoint
template <int C>
struct BwdSmem {
    static constexpr uint32_t TILE = (C / 64) * kAtom;
    static constexpr uint32_t Q = 0;               // qh [128 q x C]
    static constexpr uint32_t DO = Q + TILE;        // dO [128 q x C]
    static constexpr uint32_t F = DO + TILE;        // feature ring [2]
    static constexpr uint32_t PSI = F + 2 * TILE;   // psi [1]
    static constexpr uint32_t P = PSI + TILE;       // P  [128 q x 128 j]
    static constexpr uint32_t E = P + 2 * kAtom;    // dE [128 q x 128 j]
    static constexpr uint32_t BYTES = E + 2 * kAtom;
};

// TMEM columns of the adjoint: S / dK at 0, dP / dV at 128, dqh at 256
template <int C>
__global__ void __launch_bounds__(kAThreads, 1)
    attn_bwd_kernel(const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_q,
                    const __grid_constant__ CUtensorMap map_do, AttnParams p)
{
    using L = BwdSmem<C>;
    constexpr int A = C / 64;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sb = smem_u32(base);
    __shared__ uint64_t f_full[2], f_empty[2], psi_full, psi_empty, s_full, pe_full, x_full, x_empty, m_full[4];
    __shared__ uint64_t q_bar, drain_bar;
    __shared__ uint32_t mask[4][4];
    __shared__ float wk[C / 6 + 2];
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    __shared__ AttnCam cam_s;

    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    if (tid < static_cast<int>(sizeof(AttnCam) / 4))
        reinterpret_cast<float *>(&cam_s)[tid] = reinterpret_cast<const float *>(p.camd)[tid];
    const int t0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * p.n_tiles / gridDim.x);
    const int t1 = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * p.n_tiles / gridDim.x);
    const int nt = t1 - t0;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&f_full[i], 1);
            mbar_init(&f_empty[i], 1);
        }
        mbar_init(&psi_full, 4);
        mbar_init(&psi_empty, 1);
        mbar_init(&s_full, 1);
        mbar_init(&pe_full, 4);
        mbar_init(&x_full, 1);
        mbar_init(&x_empty, 4);
        for (int i = 0; i < 4; ++i) mbar_init(&m_full[i], 4);
        mbar_init(&q_bar, 1);
        mbar_init(&drain_bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    for (int k = tid; k < C / 6 + 2; k += kAThreads)
        wk[k] = expf(-kLnB * 6.0f * static_cast<float>(k) / static_cast<float>(C));
    if (wid == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    DevStatus *st = p.status;

    if (wid == 0) {
        // ---------------- TMA producer: qh and dO once, then the feature tiles
        int issued = 0, landed_q = 0;
        if (lane == 0 && nt > 0) {
            mbar_arrive_expect_tx(&q_bar, 2 * L::TILE);
            for (int a = 0; a < A; ++a) {
                tma_load_2d(base + L::Q + a * kAtom, &map_q, a * 64, 0, &q_bar);
                tma_load_2d(base + L::DO + a * kAtom, &map_do, a * 64, 0, &q_bar);
            }
            landed_q = 1;
            for (int t = 0; t < nt; ++t) {
                const int s = t & 1;
                if (t >= 2 && !await(&f_empty[s], ((t >> 1) - 1) & 1, st, kSiteDecodeLoad, &abort_flag)) break;
                mbar_arrive_expect_tx(&f_full[s], L::TILE);
                for (int a = 0; a < A; ++a)
                    tma_load_2d(base + L::F + s * L::TILE + a * kAtom, &map_f, a * 64, (t0 + t) * kAT, &f_full[s]);
                ++issued;
            }
            if (landed_q) mbar_wait(&q_bar, 0, st, kSiteDrain);
            for (int t = (issued > 2 ? issued - 2 : 0); t < issued; ++t) mbar_wait(&f_full[t & 1], (t >> 1) & 1, st, kSiteDrain);
        }
    } else if (wid == 1) {
        // ---------------- MMA issuer
        if (lane == 0 && nt > 0) {
            const uint32_t id_s = idesc_bf16(128, kAT);                 // S, dP: [q x j]
            const uint32_t id_dq = idesc_bf16(128, C) | (1u << 16);     // dqh: B = [f | psi] MN-major
            const uint32_t id_x = idesc_bf16(128, C) | (1u << 15) | (1u << 16); // dK, dV: A = dE^T / P^T, B = qh / dO, both MN-major
            bool ok = await(&q_bar, 0, st, kSiteDecodeQ, &abort_flag);
            for (int t = 0; t < nt && ok; ++t) {
                const int b = t & 1;
                ok = await(&f_full[b], (t >> 1) & 1, st, kSiteDecodeLoad, &abort_flag) &&
                     await(&psi_full, t & 1, st, kSiteDecodeMma, &abort_flag) &&
                     (t < 1 || await(&x_empty, (t - 1) & 1, st, kSiteDecodeMma, &abort_flag));
                if (!ok) break;
                tc_fence_after();
                const uint32_t fb = sb + L::F + b * L::TILE;
                // S = qh [f | psi]^T (cols 0..127), dP = dO f^T (cols 128..255)
#pragma unroll 1
                for (int k = 0; k < C / 16; ++k) {
                    const uint32_t off = (k >> 2) * kAtom + (k & 3) * 32;
                    const uint64_t aq = sw128_desc(sb + L::Q + off), ad = sw128_desc(sb + L::DO + off);
                    const uint64_t bf = sw128_desc(fb + off);
                    mma_bf16(tmem, aq, bf, id_s, k > 0 ? 1u : 0u);
                    mma_bf16(tmem, aq, sw128_desc(sb + L::PSI + off), id_s, 1u);
                    mma_bf16(tmem + 128, ad, bf, id_s, k > 0 ? 1u : 0u);
                }
                mma_commit(&s_full);
                if (!await(&pe_full, t & 1, st, kSiteDecodeMma, &abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // dqh += dE [f | psi] (over the tile's surfels)
#pragma unroll 1
                for (int k = 0; k < kAT / 16; ++k) {
                    const uint64_t a = sw128_desc(sb + L::E + (k >> 2) * kAtom + (k & 3) * 32);
                    mma_bf16(tmem + 256, a, sw128_desc_mn(fb + k * 2048, kAtom, 1024), id_dq, (t > 0 || k > 0) ? 1u : 0u);
                    mma_bf16(tmem + 256, a, sw128_desc_mn(sb + L::PSI + k * 2048, kAtom, 1024), id_dq, 1u);
                }
                mma_commit(&psi_empty);
                // dK = dE^T qh (cols 0..), dV = P^T dO (cols 128..): M = surfels, K = queries
#pragma unroll 1
                for (int k = 0; k < 128 / 16; ++k) {
                    // A [M = 128 surfels, K = 16 queries] MN-major from the [q x j] tiles: rows
                    // 16k..16k+15 (queries) of both 64-surfel atoms
                    const uint64_t ae = sw128_desc_mn(sb + L::E + k * 2048, kAtom, 1024);
                    const uint64_t ap = sw128_desc_mn(sb + L::P + k * 2048, kAtom, 1024);
                    const uint64_t bq = sw128_desc_mn(sb + L::Q + k * 2048, kAtom, 1024);
                    const uint64_t bd = sw128_desc_mn(sb + L::DO + k * 2048, kAtom, 1024);
                    mma_bf16(tmem, ae, bq, id_x, k > 0 ? 1u : 0u);
                    mma_bf16(tmem + 128, ap, bd, id_x, k > 0 ? 1u : 0u);
                }
                mma_commit(&x_full);
                mma_commit(&f_empty[b]);
            }
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, st, kSiteDrain);
        }
    } else if (is_psi_warp(wid)) {
        // ---------------- frustum mask and psi tile, one surfel per thread
        const int gq = psi_warp_index(wid), row = gq * 32 + lane;
        auto fetch = [&](int t, float *m5) {
            const int64_t j = static_cast<int64_t>(t0 + t) * kAT + row;
            const bool valid = t < nt && j < p.n;
            m5[0] = valid ? p.mu[3 * j] : 0.f;
            m5[1] = valid ? p.mu[3 * j + 1] : 0.f;
            m5[2] = valid ? p.mu[3 * j + 2] : 0.f;
            m5[3] = valid ? p.scale[2 * j] : -1.f;
            m5[4] = valid ? p.scale[2 * j + 1] : -1.f;
        };
        float nx[5];
        fetch(0, nx);
        for (int t = 0; t < nt; ++t) {
            const float mx = nx[0], my = nx[1], mz = nx[2], su = nx[3], sv = nx[4];
            fetch(t + 1, nx);
            if (t >= 1 && !await_warp(&psi_empty, (t - 1) & 1, st, kSiteDecodeMma, &abort_flag)) break;
            const bool act = su >= 0.f && frustum_active(cam_s, mx, my, mz, su, sv);
            const uint32_t word = __ballot_sync(0xffffffffu, act);
            if (lane == 0) mask[t & 3][gq] = word;
            __syncwarp();
            if (lane == 0) mbar_arrive(&m_full[t & 3]);
            psi_row<C>(sb + L::PSI, row, mx, my, mz, wk);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&psi_full);
        }
    } else {
        // ---------------- per query row: P, dE; then per surfel row: dK, dV
        const int q4 = wid & 3;
        const int row = q4 * 32 + lane;
        const uint32_t lane_bits = static_cast<uint32_t>(q4 * 32) << 16;
        const bool qvalid = row < p.n_q;
        const float Mi = qvalid ? p.M[row] : 0.0f;
        const float Li = qvalid ? p.Linv[row] : 0.0f;
        const float Di = qvalid ? p.Dq[row] : 0.0f;
        bool ok = true;
        for (int t = 0; t < nt && ok; ++t) {
            ok = await_warp(&m_full[t & 3], (t >> 2) & 1, st, kSiteDecodeMma, &abort_flag) &&
                 await_warp(&s_full, t & 1, st, kSiteDecodeMma, &abort_flag);
            if (!ok) break;
            uint32_t mw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) mw[k] = mask[t & 3][k];
            tc_fence_after();
            // P_ij and dE_ij = P_ij (dP_ij - D_i), 32 surfels at a time
#pragma unroll 1
            for (int c0 = 0; c0 < kAT; c0 += 32) {
                uint32_t s[32], g[32];
                tmem_ld16_async(tmem + lane_bits + c0, s);
                tmem_ld16_async(tmem + lane_bits + c0 + 16, s + 16);
                tmem_ld16_async(tmem + lane_bits + 128 + c0, g);
                tmem_ld16_async(tmem + lane_bits + 128 + c0 + 16, g + 16);
                tmem_wait_ld();
                const uint32_t mword = mw[c0 >> 5];
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    uint32_t wp[4], we[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        float pv[2], ev[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int jj = ch * 8 + 2 * e + h;
                            const bool a = qvalid && ((mword >> jj) & 1u);
                            pv[h] = a ? ex2f(__uint_as_float(s[jj]) * kLog2e - Mi) * Li : 0.0f;
                            ev[h] = pv[h] * (__uint_as_float(g[jj]) - Di);
                        }
                        wp[e] = pack_bf16(pv[0], pv[1]);
                        we[e] = pack_bf16(ev[0], ev[1]);
                    }
                    const int chunk = (c0 >> 3) + ch;
                    st_shared_v4(sb + L::P + tile_off(row, chunk), wp[0], wp[1], wp[2], wp[3]);
                    st_shared_v4(sb + L::E + tile_off(row, chunk), we[0], we[1], we[2], we[3]);
                }
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&pe_full);
            // per surfel (TMEM lane = surfel of the tile): dK (cols 0..C), dV (cols 128..)
            if (!(ok = await_warp(&x_full, t & 1, st, kSiteDecodeMma, &abort_flag))) break;
            tc_fence_after();
            const int64_t j = static_cast<int64_t>(t0 + t) * kAT + row;
            const bool act = (mw[row >> 5] >> (row & 31)) & 1u;
            float mj[3] = {0.f, 0.f, 0.f};
            if (act) {
                mj[0] = p.mu[3 * j];
                mj[1] = p.mu[3 * j + 1];
                mj[2] = p.mu[3 * j + 2];
            }
            // dK row in registers; dL/dmu_a = sum over k of w_k (dK[6k+a] cos(m_a w_k)
            // - dK[6k+3+a] sin(m_a w_k)) (the derivative of the psi row)
            uint32_t dk[C];
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += 16) tmem_ld16_async(tmem + lane_bits + c0, dk + c0);
            tmem_wait_ld();
            float gm[3] = {0.f, 0.f, 0.f};
            if (act && p.g_mu) {
#pragma unroll
                for (int k = 0; 6 * k < C; ++k) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float sn, cs;
                        __sincosf(mj[a] * wk[k], &sn, &cs);
                        if (6 * k + a < C) gm[a] = fmaf(__uint_as_float(dk[6 * k + a]) * wk[k], cs, gm[a]);
                        if (6 * k + 3 + a < C) gm[a] = fmaf(-__uint_as_float(dk[6 * k + 3 + a]) * wk[k], sn, gm[a]);
                    }
                }
            }
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += 16) {
                uint32_t dv[16];
                tmem_ld16_async(tmem + lane_bits + 128 + c0, dv);
                tmem_wait_ld();
                if (act && p.g_feat) {
                    // added with 16-byte reductions: no load of the row to wait for
                    float4 *gf = reinterpret_cast<float4 *>(p.g_feat + j * C + c0);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        atomicAdd(gf + e, make_float4(__uint_as_float(dk[c0 + 4 * e]) + __uint_as_float(dv[4 * e]),
                                                      __uint_as_float(dk[c0 + 4 * e + 1]) + __uint_as_float(dv[4 * e + 1]),
                                                      __uint_as_float(dk[c0 + 4 * e + 2]) + __uint_as_float(dv[4 * e + 2]),
                                                      __uint_as_float(dk[c0 + 4 * e + 3]) + __uint_as_float(dv[4 * e + 3])));
                }
            }
            if (act && p.g_mu) {
                atomicAdd(p.g_mu + 3 * j, gm[0]);
                atomicAdd(p.g_mu + 3 * j + 1, gm[1]);
                atomicAdd(p.g_mu + 3 * j + 2, gm[2]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&x_empty);
        }
        // dqh partial of this CTA (query rows)
        if (ok && nt > 0) {
            // the last tile's MMAs (x_full) include the dqh accumulation
            tc_fence_after();
            float *dst = p.part_dq + (static_cast<int64_t>(blockIdx.x) * 128 + row) * C;
#pragma unroll 1
            for (int c0 = 0; c0 < C; c0 += 16) {
                uint32_t o[16];
                tmem_ld16_async(tmem + lane_bits + 256 + c0, o);
                tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; e += 4)
                    *reinterpret_cast<float4 *>(dst + c0 + e) =
                        make_float4(__uint_as_float(o[e]), __uint_as_float(o[e + 1]), __uint_as_float(o[e + 2]),
                                    __uint_as_float(o[e + 3]));
            }
        } else {
            float *dst = p.part_dq + (static_cast<int64_t>(blockIdx.x) * 128 + row) * C;
            for (int c = 0; c < C; ++c) dst[c] = 0.0f;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

// ------------------------------------------------------------------ small kernels
// qh = (Q W_Q) W_K^T / sqrt(d) in FP32 and as the padded BF16 A tile [128 x C]
// (rows >= n_q zero); q = Q W_Q kept for the adjoint. One CTA per row.
__global__ void __launch_bounds__(256) attn_qh_kernel(const float *Q, int n_q, const float *WQ, const float *WK, int C,
                                                      int d, float *q, float *qh, __nv_bfloat16 *qh_bf, AttnCam cam,
                                                      AttnCam *cam_out)
{
    __shared__ float qs[256];
    const int i = blockIdx.x;
    if (i == 0 && threadIdx.x == 0) *cam_out = cam;
    if (i >= n_q) {
        for (int c = threadIdx.x; c < C; c += blockDim.x) qh_bf[i * C + c] = __float2bfloat16_rn(0.0f);
        return;
    }
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < C; ++c) acc = fmaf(Q[i * C + c], WQ[c * d + e], acc);
        qs[e] = acc;
        q[i * d + e] = acc;
    }
    __syncthreads();
    const float inv = rsqrtf(static_cast<float>(d));
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float acc = 0.0f;
        for (int e = 0; e < d; ++e) acc = fmaf(qs[e], WK[c * d + e], acc);
        acc *= inv;
        qh[i * C + c] = acc;
        qh_bf[i * C + c] = __float2bfloat16_rn(acc);
    }
}

// Merge the per-CTA partials of query i: M = max_g m_g, L = sum_g l_g 2^(m_g -
// M), O = sum_g O_g 2^(m_g - M) / L (zero without active surfels), out = O W_V.
__global__ void __launch_bounds__(256) attn_combine_kernel(const float *part_m, const float *part_l,
                                                           const float *part_o, int G, int C, int d, const float *WV,
                                                           float *out, float *O, float *M, float *Linv)
{
    __shared__ float os[256];
    __shared__ float Mmax, Ls;
    const int i = blockIdx.x;
    if (threadIdx.x == 0) {
        float m = -__int_as_float(0x7f800000);
        for (int g = 0; g < G; ++g) m = fmaxf(m, part_m[g * 128 + i]);
        float l = 0.0f;
        if (m > -__int_as_float(0x7f800000))
            for (int g = 0; g < G; ++g)
                if (part_l[g * 128 + i] > 0.0f) l += part_l[g * 128 + i] * exp2f(part_m[g * 128 + i] - m);
        Mmax = m;
        Ls = l;
        M[i] = m;
        Linv[i] = l > 0.0f ? 1.0f / l : 0.0f;
    }
    __syncthreads();
    const float m = Mmax, inv = Ls > 0.0f ? 1.0f / Ls : 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float acc = 0.0f;
        if (inv > 0.0f)
            for (int g = 0; g < G; ++g) {
                const float l = part_l[g * 128 + i];
                if (l > 0.0f) acc += part_o[(static_cast<int64_t>(g) * 128 + i) * C + c] * exp2f(part_m[g * 128 + i] - m);
            }
        acc *= inv;
        os[c] = acc;
        O[i * C + c] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < C; ++c) acc = fmaf(os[c], WV[c * d + e], acc);
        out[i * d + e] = acc;
    }
}

// Adjoint set-up for query i: dO = G W_V^T, D = dO . O (the forward's
// normalised O), dO as the padded BF16 tile (rows >= n_q zero).
__global__ void __launch_bounds__(256) attn_bwd_prep_kernel(const float *G, int n_q, const float *WV, const float *O,
                                                            int C, int d, float *dO, float *Dq,
                                                            __nv_bfloat16 *dO_bf)
{
    __shared__ float red[8];
    const int i = blockIdx.x;
    if (i >= n_q) {
        for (int c = threadIdx.x; c < C; c += blockDim.x) dO_bf[i * C + c] = __float2bfloat16_rn(0.0f);
        return;
    }
    float part = 0.0f;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float acc = 0.0f;
        for (int e = 0; e < d; ++e) acc = fmaf(G[i * d + e], WV[c * d + e], acc);
        dO[i * C + c] = acc;
        dO_bf[i * C + c] = __float2bfloat16_rn(acc);
        part = fmaf(acc, O[i * C + c], part);
    }
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (static_cast<int>(blockDim.x) >> 5); ++w) s += red[w];
        Dq[i] = s;
    }
}

// The adjoint's small products, one CTA per output row:
//   dqh = sum_g dqh_g,  dq = dqh W_K / sqrt(d),  dQ = dq W_Q^T
// (rows of dQ), then dW_Q = Q^T dq, dW_K = dqh^T q / sqrt(d), dW_V = O^T G
// (rows c of the [C x d] gradients).
__global__ void __launch_bounds__(256) attn_bwd_q_kernel(const float *part_dq, int G, int n_q, int C, int d,
                                                         const float *WK, const float *WQ, float *dqh, float *dq,
                                                         float *gQ)
{
    __shared__ float hs[256], qs[256];
    const int i = blockIdx.x;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float acc = 0.0f;
        for (int g = 0; g < G; ++g) acc += part_dq[(static_cast<int64_t>(g) * 128 + i) * C + c];
        hs[c] = acc;
        dqh[i * C + c] = acc;
    }
    __syncthreads();
    const float inv = rsqrtf(static_cast<float>(d));
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float acc = 0.0f;
        for (int c = 0; c < C; ++c) acc = fmaf(hs[c], WK[c * d + e], acc);
        acc *= inv;
        qs[e] = acc;
        dq[i * d + e] = acc;
    }
    __syncthreads();
    if (gQ)
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            float acc = 0.0f;
            for (int e = 0; e < d; ++e) acc = fmaf(qs[e], WQ[c * d + e], acc);
            gQ[i * C + c] = acc;
        }
}

__global__ void __launch_bounds__(256) attn_bwd_w_kernel(const float *Q, const float *q, const float *dq,
                                                         const float *dqh, const float *O, const float *G, int n_q,
                                                         int C, int d, float *gWQ, float *gWK, float *gWV)
{
    const int c = blockIdx.x;
    const float inv = rsqrtf(static_cast<float>(d));
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        float wq = 0.0f, wk = 0.0f, wv = 0.0f;
        for (int i = 0; i < n_q; ++i) {
            wq = fmaf(Q[i * C + c], dq[i * d + e], wq);
            wk = fmaf(dqh[i * C + c], q[i * d + e], wk);
            wv = fmaf(O[i * C + c], G[i * d + e], wv);
        }
        if (gWQ) gWQ[c * d + e] = wq;
        if (gWK) gWK[c * d + e] = wk * inv;
        if (gWV) gWV[c * d + e] = wv;
    }
}

// ------------------------------------------------------------------ workspace
struct AttnWs {
    AttnCam *cam;
    float *q, *qh, *O, *M, *Linv, *dO, *Dq, *dqh, *dq;
    __nv_bfloat16 *qh_bf, *dO_bf;
    float *part_m, *part_l, *part_o;
};

int attn_grid(int64_t n)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (std::max<int64_t>(n, 1) + kAT - 1) / kAT;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(tiles, sms)));
}

constexpr int kMaxGrid = 1024; // partial slots (>= SMs of any device this runs on)

AttnWs carve(void *ws, int C, int d)
{
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t bytes) {
        char *r = p;
        p += up(bytes);
        return r;
    };
    AttnWs w;
    w.cam = reinterpret_cast<AttnCam *>(take(sizeof(AttnCam)));
    w.q = reinterpret_cast<float *>(take(128 * d * 4));
    w.qh = reinterpret_cast<float *>(take(128 * C * 4));
    w.O = reinterpret_cast<float *>(take(128 * C * 4));
    w.M = reinterpret_cast<float *>(take(128 * 4));
    w.Linv = reinterpret_cast<float *>(take(128 * 4));
    w.dO = reinterpret_cast<float *>(take(128 * C * 4));
    w.Dq = reinterpret_cast<float *>(take(128 * 4));
    w.dqh = reinterpret_cast<float *>(take(128 * C * 4));
    w.dq = reinterpret_cast<float *>(take(128 * d * 4));
    w.qh_bf = reinterpret_cast<__nv_bfloat16 *>(take(128 * C * 2));
    w.dO_bf = reinterpret_cast<__nv_bfloat16 *>(take(128 * C * 2));
    w.part_m = reinterpret_cast<float *>(take(kMaxGrid * 128 * 4));
    w.part_l = reinterpret_cast<float *>(take(kMaxGrid * 128 * 4));
    w.part_o = reinterpret_cast<float *>(take(static_cast<size_t>(kMaxGrid) * 128 * C * 4));
    return w;
}

AttnCam make_cam(const psi_camera &cam, float z_near)
{
    AttnCam a{};
    for (int i = 0; i < 9; ++i) a.R[i] = cam.R[i];
    for (int i = 0; i < 3; ++i) a.t[i] = cam.t[i];
    a.fx = cam.fx;
    a.fy = cam.fy;
    a.cx = cam.cx;
    a.cy = cam.cy;
    a.W = static_cast<float>(cam.width);
    a.H = static_cast<float>(cam.height);
    a.z_near = z_near;
    return a;
}

template <class Smem>
size_t smem_bytes()
{
    return Smem::BYTES + 1024;
}

} // namespace

size_t attention_workspace_bytes(int64_t n, int C, int d, int n_q)
{
    (void)n;
    (void)n_q;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    return up(sizeof(AttnCam)) + up(128 * d * 4) * 2 + up(128 * C * 4) * 4 + up(128 * 4) * 3 + up(128 * C * 2) * 2 +
           up(kMaxGrid * 128 * 4) * 2 + up(static_cast<size_t>(kMaxGrid) * 128 * C * 4) + 256;
}

cudaError_t launch_attention(const psi_surfels &s, const void *feat, int C, const psi_camera &cam, float z_near,
                             const float *Q, int n_q, const float *WQ, const float *WK, const float *WV, int d,
                             float *out, void *ws, DevStatus *status, cudaStream_t st, const char **why)
{
    const AttnWs w = carve(ws, C, d);
    attn_qh_kernel<<<128, 256, 0, st>>>(Q, n_q, WQ, WK, C, d, w.q, w.qh, w.qh_bf, make_cam(cam, z_near), w.cam);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t N = s.n;
    const int G = attn_grid(N);
    CUtensorMap map_f, map_q;
    if (!encode_2d_bf16(&map_f, feat, static_cast<uint64_t>(C), static_cast<uint64_t>(std::max<int64_t>(N, 1)), 64, kAT) ||
        !encode_2d_bf16(&map_q, w.qh_bf, static_cast<uint64_t>(C), 128, 64, 128)) {
        *why = "cuTensorMapEncodeTiled failed";
        return cudaErrorInvalidValue;
    }
    AttnParams p{};
    p.n = N;
    p.n_tiles = static_cast<int>((N + kAT - 1) / kAT);
    p.n_q = n_q;
    p.camd = w.cam;
    p.mu = s.mu;
    p.scale = s.scale;
    p.part_m = w.part_m;
    p.part_l = w.part_l;
    p.part_o = w.part_o;
    p.status = status;
    if (N > 0) {
        if (C == 64) {
            const size_t sm = smem_bytes<FwdSmem<64>>();
            e = cudaFuncSetAttribute(attn_fwd_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
            if (e == cudaSuccess) attn_fwd_kernel<64><<<G, kAThreads, sm, st>>>(map_f, map_q, p);
        } else {
            const size_t sm = smem_bytes<FwdSmem<128>>();
            e = cudaFuncSetAttribute(attn_fwd_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
            if (e == cudaSuccess) attn_fwd_kernel<128><<<G, kAThreads, sm, st>>>(map_f, map_q, p);
        }
        if (e != cudaSuccess) return e;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    attn_combine_kernel<<<n_q, 256, 0, st>>>(w.part_m, w.part_l, w.part_o, N > 0 ? G : 0, C, d, WV, out, w.O, w.M,
                                             w.Linv);
    return cudaGetLastError();
}

cudaError_t launch_attention_bwd(const psi_surfels &s, const void *feat, int C, const float *Q, int n_q, const float *WQ, const float *WK, const float *WV, int d,
                                 const float *G_out, float *gQ, float *gWQ, float *gWK, float *gWV, float *g_feat,
                                 float *g_mu, void *ws, DevStatus *status, cudaStream_t st, const char **why)
{
    const AttnWs w = carve(ws, C, d);
    attn_bwd_prep_kernel<<<128, 256, 0, st>>>(G_out, n_q, WV, w.O, C, d, w.dO, w.Dq, w.dO_bf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t N = s.n;
    const int G = attn_grid(N);
    CUtensorMap map_f, map_q, map_do;
    if (!encode_2d_bf16(&map_f, feat, static_cast<uint64_t>(C), static_cast<uint64_t>(std::max<int64_t>(N, 1)), 64, kAT) ||
        !encode_2d_bf16(&map_q, w.qh_bf, static_cast<uint64_t>(C), 128, 64, 128) ||
        !encode_2d_bf16(&map_do, w.dO_bf, static_cast<uint64_t>(C), 128, 64, 128)) {
        *why = "cuTensorMapEncodeTiled failed";
        return cudaErrorInvalidValue;
    }
    AttnParams p{};
    p.n = N;
    p.n_tiles = static_cast<int>((N + kAT - 1) / kAT);
    p.n_q = n_q;
    p.camd = w.cam;
    p.mu = s.mu;
    p.scale = s.scale;
    p.M = w.M;
    p.Linv = w.Linv;
    p.Dq = w.Dq;
    p.part_dq = w.part_o; // the forward's O partials are no longer needed
    p.g_feat = g_feat;
    p.g_mu = g_mu;
    p.status = status;
    if (N > 0) {
        if (C == 64) {
            const size_t sm = smem_bytes<BwdSmem<64>>();
            e = cudaFuncSetAttribute(attn_bwd_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
            if (e == cudaSuccess) attn_bwd_kernel<64><<<G, kAThreads, sm, st>>>(map_f, map_q, map_do, p);
        } else {
            const size_t sm = smem_bytes<BwdSmem<128>>();
            e = cudaFuncSetAttribute(attn_bwd_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
            if (e == cudaSuccess) attn_bwd_kernel<128><<<G, kAThreads, sm, st>>>(map_f, map_q, map_do, p);
        }
        if (e != cudaSuccess) return e;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else {
        e = cudaMemsetAsync(w.part_o, 0, static_cast<size_t>(128) * C * 4, st);
        if (e != cudaSuccess) return e;
    }
    attn_bwd_q_kernel<<<n_q, 256, 0, st>>>(w.part_o, N > 0 ? G : 1, n_q, C, d, WK, WQ, w.dqh, w.dq, gQ);
    attn_bwd_w_kernel<<<C, 256, 0, st>>>(Q, w.q, w.dq, w.dqh, w.O, G_out, n_q, C, d, gWQ, gWK, gWV);
    return cudaGetLastError();
}

} // namespace psi
