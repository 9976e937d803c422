// Float32 binning decisions with an explicit operation order.
//
// Culling, the support radius, the ellipse bounds of the projected covariance
// (Sec. 5, Precise Tile Intersection), the tile rectangle of each mode and the
// exact ellipse-versus-tile-row test are integer decisions taken in float32.
// Every product, sum, quotient and square root below is a separately rounded
// IEEE operation (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn) and every fused
// multiply-add is an explicit __fmaf_rn, so the compiler cannot contract or
// reorder them and the tile lists are reproducible bit for bit from the
// written sequence.
#pragma once

#include "common.cuh"

namespace psi {
namespace disc {

__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kBinInflate = 1.0f + 1.0f / 1024.0f; // binning disc radius^2 factor
constexpr float kFltMax = 3.402823466e+38f;

// Smallest squared radius beyond which o * exp(-d2/2) < 1/255, rounded up:
// 2 ln(255 o) + 1e-3, with ln(x) = e ln2 + 2 atanh(s), x = m 2^e,
// m in [sqrt(1/2), sqrt(2)], s = (m-1)/(m+1), atanh by its Taylor series
// through s^9 (truncation < 1e-9).
__device__ __forceinline__ float opacity_radius2(float o)
{
    const float x = mul(255.0f, o);
    if (!(x > 1.0f)) return 1e-3f;
    const uint32_t b = __float_as_uint(x);
    int e = static_cast<int>(b >> 23) - 127;
    float m = __uint_as_float((b & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) {
        m = mul(m, 0.5f);
        e = e + 1;
    }
    const float s = div(sub(m, 1.0f), add(m, 1.0f));
    const float s2 = mul(s, s);
    float p = 1.0f / 9.0f;
    p = fma(p, s2, 1.0f / 7.0f);
    p = fma(p, s2, 1.0f / 5.0f);
    p = fma(p, s2, 1.0f / 3.0f);
    p = fma(p, s2, 1.0f);
    const float lnx = fma(static_cast<float>(e), 0x1.62e430p-1f, mul(mul(2.0f, s), p));
    return fma(2.0f, lnx, 1e-3f);
}

// Result of the binning setup of one (view, surfel) record.
struct Bin {
    float ex, ey;          // ellipse centre (pixels)
    float A00, A01, A11;   // ellipse shape matrix at the binning radius
    int px0, px1, py0, py1; // rectangle of pixel indices whose centres may be covered
    float p0x, p0y;        // projected centre (pixels)
    float rd2;             // low-pass disc 2|x - p0|^2 <= r_b^2 as radius^2 in pixels; < 0: no filter
};

// x of the ellipse boundary on the line y = ey + dy (left or right branch)
__device__ __forceinline__ float chord_x(const Bin &b, float det, float dy, bool right)
{
    const float t1 = mul(b.A01, dy);
    const float t2 = fma(-dy, dy, b.A11);
    const float t3 = sqrt(fmaxf(mul(det, t2), 0.0f));
    return add(b.ex, div(right ? add(t1, t3) : sub(t1, t3), b.A11));
}

// Tile columns [c0, c1] touched in tile row ty (EXACT: only tiles whose
// pixel-centre columns meet the ellipse within the row's pixel-centre band;
// other modes: the whole rectangle). Returns false if the row has none.
__device__ __forceinline__ bool row_tiles(const Bin &b, int mode, int ty, int tw, int th, int &c0, int &c1)
{
    if (mode != PSI_ISECT_EXACT || !(b.A00 > 0.0f && b.A11 > 0.0f)) {
        c0 = b.px0 / tw;
        c1 = b.px1 / tw;
        return true;
    }
    const int r0 = max(b.py0, ty * th);
    const int r1 = min(b.py1, ty * th + th - 1);
    const float d0 = sub(add(static_cast<float>(r0), 0.5f), b.ey);
    const float d1 = sub(add(static_cast<float>(r1), 0.5f), b.ey);
    const float det = fmaxf(fma(b.A00, b.A11, -mul(b.A01, b.A01)), 0.0f);
    const float hx = sqrt(fmaxf(b.A00, 0.0f));
    const float sl = div(b.A01, hx); // dy of the rightmost point; the leftmost is at -sl
    float xmin, xmax;
    const float yl = -sl;
    if (yl < d0)
        xmin = chord_x(b, det, d0, false);
    else if (yl > d1)
        xmin = chord_x(b, det, d1, false);
    else
        xmin = sub(b.ex, hx);
    const float yr = sl;
    if (yr < d0)
        xmax = chord_x(b, det, d0, true);
    else if (yr > d1)
        xmax = chord_x(b, det, d1, true);
    else
        xmax = add(b.ex, hx);
    float fl = ceilf(sub(xmin, 0.5f));
    float fh = floorf(sub(xmax, 0.5f));
    fl = fmaxf(fl, static_cast<float>(b.px0));
    fh = fminf(fh, static_cast<float>(b.px1));
    bool ok = fl <= fh;
    if (b.rd2 >= 0.0f) {
        // low-pass disc: its chord at the band's row nearest to the centre; the
        // row's columns are the hull of both ranges
        const float lo = add(static_cast<float>(r0), 0.5f), hi = add(static_cast<float>(r1), 0.5f);
        const float dy = b.p0y < lo ? sub(lo, b.p0y) : (b.p0y > hi ? sub(b.p0y, hi) : 0.0f);
        const float tt = fma(-dy, dy, b.rd2);
        if (tt >= 0.0f) {
            const float h = sqrt(tt);
            float gl = ceilf(sub(sub(b.p0x, h), 0.5f));
            float gh = floorf(sub(add(b.p0x, h), 0.5f));
            gl = fmaxf(gl, static_cast<float>(b.px0));
            gh = fminf(gh, static_cast<float>(b.px1));
            if (gl <= gh) {
                fl = ok ? fminf(fl, gl) : gl;
                fh = ok ? fmaxf(fh, gh) : gh;
                ok = true;
            }
        }
    }
    if (!ok) return false;
    c0 = static_cast<int>(fl) / tw;
    c1 = static_cast<int>(fh) / tw;
    return true;
}

// Bin records are 32 bytes: ex, ey, A00, A01, A11, depth, px0|px1<<16,
// py0|py1<<16; with the low-pass filter 48 bytes: then p0x, p0y, rd2, 0.
__device__ __forceinline__ int bin_stride(bool lowpass) { return lowpass ? 3 : 2; } // float4 per record

__device__ __forceinline__ void store_bin(float4 *dst, const Bin &b, float depth, bool lowpass)
{
    dst[0] = make_float4(b.ex, b.ey, b.A00, b.A01);
    dst[1] = make_float4(b.A11, depth, __uint_as_float(static_cast<uint32_t>(b.px0) | (static_cast<uint32_t>(b.px1) << 16)),
                         __uint_as_float(static_cast<uint32_t>(b.py0) | (static_cast<uint32_t>(b.py1) << 16)));
    if (lowpass) dst[2] = make_float4(b.p0x, b.p0y, b.rd2, 0.0f);
}

__device__ __forceinline__ Bin load_bin(const float4 *src, float &depth, bool lowpass)
{
    const float4 a = src[0], c = src[1];
    Bin b;
    if (lowpass) {
        const float4 l = src[2];
        b.p0x = l.x;
        b.p0y = l.y;
        b.rd2 = l.z;
    } else {
        b.p0x = b.p0y = 0.0f;
        b.rd2 = -1.0f;
    }
    b.ex = a.x;
    b.ey = a.y;
    b.A00 = a.z;
    b.A01 = a.w;
    b.A11 = c.x;
    depth = c.y;
    const uint32_t px = __float_as_uint(c.z), py = __float_as_uint(c.w);
    b.px0 = static_cast<int>(px & 0xFFFFu);
    b.px1 = static_cast<int>(px >> 16);
    b.py0 = static_cast<int>(py & 0xFFFFu);
    b.py1 = static_cast<int>(py >> 16);
    return b;
}

__device__ __forceinline__ uint32_t count_tiles(const Bin &b, int mode, int tw, int th)
{
    uint32_t c = 0;
    const int ty0 = b.py0 / th, ty1 = b.py1 / th;
    if (mode != PSI_ISECT_EXACT) return static_cast<uint32_t>((b.px1 / tw - b.px0 / tw + 1) * (ty1 - ty0 + 1));
    for (int ty = ty0; ty <= ty1; ++ty) {
        int c0, c1;
        if (row_tiles(b, mode, ty, tw, th, c0, c1)) c += static_cast<uint32_t>(c1 - c0 + 1);
    }
    return c;
}

} // namespace disc
} // namespace psi
