/*
 * psi_oracle.c -- plain, slow CPU reference for the surfel rendering path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library links or calls this file;
 * only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it. It shares no code, header or constant table with the CUDA path.
 *
 * Two independent parts:
 *
 *  (1) The discrete path (pinned FP32). Culling, support radius, ellipse
 *      bounds, tile rectangles, the exact ellipse-vs-tile test and the sort
 *      keys are integer decisions taken in float32. This part spells out the
 *      float32 operation sequence explicitly (fmaf where an FMA is specified,
 *      everything else separately rounded; the file is compiled with
 *      -ffp-contract=off), so that tile lists and key arrays can be compared
 *      bit for bit. The written sequence is the reading of Sec. 5 "Precise
 *      Tile Intersection" (the AABB half-widths from the projected covariance)
 *      plus the exact ellipse test, stated in the design notes.
 *
 *  (2) The value path (FP64). For every pixel it walks ALL non-culled surfels
 *      in canonical depth order (no tiles), intersects the pixel ray with each
 *      surfel plane by solving a 3x3 linear system with partial pivoting
 *      (the 2D-surfel ray-splat intersection of Sec. 3.1, written as linear
 *      algebra), evaluates alpha = o * exp(-(u^2+v^2)/2) (Sec. 3.1), blends
 *      front to back with Eq. (1), and selects the Top-K weights
 *      omega_j = alpha_j * prod_{k<j}(1 - alpha_k) for the feature sum of the
 *      Top-K Hard Selection equation (Sec. 5). The gradient is the closed form
 *      of the blending adjoint with suffix sums plus implicit differentiation
 *      of the ray-plane solve.
 *
 * Optional 2DGS object-space low-pass filter (the surfel model of Sec. 3.1
 * follows 2D Gaussian Splatting): with it the Gaussian argument is
 * rho = min(u^2+v^2, 2 |x - c|^2), c the pixel position of the projected
 * centre, i.e. the larger of the surfel's value and that of a screen-space
 * Gaussian of standard deviation sqrt(2)/2 pixel at c, so a surfel seen edge
 * on still covers about one pixel. The support becomes rho <= r^2; binning
 * covers the ellipse and the disc 2 |x - c|^2 <= r_b^2.
 *
 * Conventions: OpenCV camera (x right, y down, z forward), x_c = R x_w + t,
 * pixel (px,py) samples (px+1/2, py+1/2). Thresholds: alpha < 1/255 skipped,
 * alpha clamped to 0.99, stop after the surfel that takes T below T_eps.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* (1) discrete path, float32                                          */
/* ------------------------------------------------------------------ */

enum { OR_SPHERE = 0, OR_AABB = 1, OR_EXACT = 2 };

/* OR_PLANT selects a deliberately wrong variant, built only by the test that
 * checks that the pins catch it: 1 drops the 1/2 in the Gaussian, 2 updates T
 * before taking the weight, 3 keeps the K smallest weights, 4 flips the sign
 * of the centre gradient, 5 mirrors the exact-test chord, 6 drops the factor 2
 * of the low-pass term, 7 flips the sign of its centre gradient, 8 tests only
 * the centre's depth against the near plane, 9 takes the smaller eigenvalue
 * for the SPHERE radius, 10 tests the unit disc instead of the binning disc
 * against the near plane. 0 = correct. */
#ifndef OR_PLANT
#define OR_PLANT 0
#endif

static float f_bits_to_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t f_float_to_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* Upper bound of 2*ln(255*o): the squared radius beyond which
 * o*exp(-d2/2) < 1/255. ln(x) = e*ln2 + ln(m) with x = m*2^e,
 * m in [sqrt(1/2), sqrt(2)], and ln(m) = 2*atanh(s) = 2(s + s^3/3 + s^5/5 +
 * s^7/7 + s^9/9 + ...), s = (m-1)/(m+1) (Taylor series of atanh). Truncation
 * error < 1e-9; float rounding < 1e-5; a margin of 1e-3 makes it an upper
 * bound. */
static float rho_opacity(float o)
{
    float x = 255.0f * o;
    if (!(x > 1.0f)) return 1e-3f; /* 2 ln(x) <= 2e-7 here */
    uint32_t b = f_float_to_bits(x);
    int e = (int)(b >> 23) - 127;
    float m = f_bits_to_float((b & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 1.0f / 9.0f;
    p = fmaf(p, s2, 1.0f / 7.0f);
    p = fmaf(p, s2, 1.0f / 5.0f);
    p = fmaf(p, s2, 1.0f / 3.0f);
    p = fmaf(p, s2, 1.0f);
    float lnx = fmaf((float)e, 0x1.62e430p-1f, (2.0f * s) * p);
    return fmaf(2.0f, lnx, 1e-3f);
}

typedef struct {
    int ok;                 /* 1 = visible and touching at least one pixel centre */
    float r2;               /* support radius^2 used by the per-pixel test */
    float depth;            /* camera-space z of the centre (sort key) */
    float ex, ey;           /* ellipse centre (pixels) */
    float A00, A01, A11;    /* ellipse shape matrix (binning radius) */
    float hx, hy;           /* exact AABB half-widths */
    float extx, exty;       /* half-extents used for the rectangle (mode) */
    int px0, px1, py0, py1; /* pixel-index rectangle of covered pixel centres */
    float p0x, p0y;         /* projected centre (pixels) */
    float rd2;              /* low-pass disc radius^2 in pixels (binning), < 0: no filter */
} disc_t;

/* camera: R[9] row-major, t[3], fx, fy, cx, cy, W, H (all float) */
static void disc_surfel(const float *mu, const float *tu, const float *tv, float su, float sv, float o,
                        const float *cam, float chi2, float znear, int oprad, int mode, int lowpass, disc_t *d)
{
    const float *R = cam, *t = cam + 9;
    const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const int W = (int)cam[16], H = (int)cam[17];
    memset(d, 0, sizeof(*d));

    /* camera-space centre and scaled tangent axes */
    float xc[3], uu[3], vv[3];
    for (int k = 0; k < 3; k++) {
        xc[k] = fmaf(R[3 * k + 2], mu[2], fmaf(R[3 * k + 1], mu[1], fmaf(R[3 * k + 0], mu[0], t[k])));
        float au = fmaf(R[3 * k + 2], tu[2], fmaf(R[3 * k + 1], tu[1], R[3 * k + 0] * tu[0]));
        float av = fmaf(R[3 * k + 2], tv[2], fmaf(R[3 * k + 1], tv[1], R[3 * k + 0] * tv[0]));
        uu[k] = su * au;
        vv[k] = sv * av;
    }
    if (!(o >= 1.0f / 255.0f)) return;

    float r2 = chi2;
    if (oprad) r2 = fminf(chi2, rho_opacity(o));
    const float r2b = r2 * (1.0f + 1.0f / 1024.0f); /* binning radius^2 */

    /* near-plane cull of the whole binning disc */
    const float w = xc[2];
    const float nab = sqrtf(fmaf(uu[2], uu[2], vv[2] * vv[2]));
    const float rb = sqrtf(r2b);
    float zmin = fmaf(-rb, nab, w);
    if (OR_PLANT == 8) zmin = w;            /* planted: centre-only near test */
    if (OR_PLANT == 10) zmin = w - nab;     /* planted: unit disc instead of the binning disc */
    if (!(zmin > znear)) return;

    /* pixel-homogeneous columns, shifted so the projected centre is the origin */
    const float mcx = fmaf(fx, xc[0], cx * xc[2]);
    const float mcy = fmaf(fy, xc[1], cy * xc[2]);
    const float p0x = mcx / w, p0y = mcy / w;
    float mu_[3], mv_[3], mc_[3];
    mu_[0] = fmaf(-p0x, uu[2], fmaf(fx, uu[0], cx * uu[2]));
    mu_[1] = fmaf(-p0y, uu[2], fmaf(fy, uu[1], cy * uu[2]));
    mu_[2] = uu[2];
    mv_[0] = fmaf(-p0x, vv[2], fmaf(fx, vv[0], cx * vv[2]));
    mv_[1] = fmaf(-p0y, vv[2], fmaf(fy, vv[1], cy * vv[2]));
    mv_[2] = vv[2];
    mc_[0] = fmaf(-p0x, w, mcx);
    mc_[1] = fmaf(-p0y, w, mcy);
    mc_[2] = w;

    /* dual conic C = M diag(r2b, r2b, -1) M^T (upper triangle) */
#define CONIC(i, j) fmaf(r2b, fmaf(mu_[i], mu_[j], mv_[i] * mv_[j]), -(mc_[i] * mc_[j]))
    const float C00 = CONIC(0, 0), C01 = CONIC(0, 1), C02 = CONIC(0, 2);
    const float C11 = CONIC(1, 1), C12 = CONIC(1, 2), C22 = CONIC(2, 2);
#undef CONIC
    if (!(C22 < 0.0f)) return;

    const float ex = p0x + C02 / C22;
    const float ey = p0y + C12 / C22;
    const float q = C22 * C22;
    const float A00 = fmaf(C02, C02, -(C00 * C22)) / q;
    const float A11 = fmaf(C12, C12, -(C11 * C22)) / q;
    const float A01 = fmaf(C02, C12, -(C01 * C22)) / q;
    const float hx = sqrtf(fmaxf(A00, 0.0f));
    const float hy = sqrtf(fmaxf(A11, 0.0f));
    float extx = hx, exty = hy;
    if (mode == OR_SPHERE) {
        const float mid = 0.5f * (A00 + A11);
        const float dd = 0.5f * (A00 - A11);
        const float lam = (OR_PLANT == 9) ? mid - sqrtf(fmaf(dd, dd, A01 * A01))  /* planted: lambda_min */
                                          : mid + sqrtf(fmaf(dd, dd, A01 * A01));
        float Rs = sqrtf(fmaxf(lam, 0.0f));
        Rs = fmaxf(Rs, fmaxf(hx, hy));
        extx = Rs;
        exty = Rs;
    }
    if (!(fabsf(ex) <= FLT_MAX && fabsf(ey) <= FLT_MAX && extx <= FLT_MAX && exty <= FLT_MAX)) return;

    float lox = ceilf((ex - extx) - 0.5f), hix = floorf((ex + extx) - 0.5f);
    float loy = ceilf((ey - exty) - 0.5f), hiy = floorf((ey + exty) - 0.5f);
    /* low-pass filter: the rectangle also covers the disc 2 |x - c|^2 <= r2b */
    const float rd2 = lowpass ? r2b * 0.5f : -1.0f;
    if (lowpass) {
        const float rd = sqrtf(rd2);
        lox = fminf(lox, ceilf((p0x - rd) - 0.5f));
        hix = fmaxf(hix, floorf((p0x + rd) - 0.5f));
        loy = fminf(loy, ceilf((p0y - rd) - 0.5f));
        hiy = fmaxf(hiy, floorf((p0y + rd) - 0.5f));
    }
    lox = fmaxf(lox, 0.0f);
    loy = fmaxf(loy, 0.0f);
    hix = fminf(hix, (float)(W - 1));
    hiy = fminf(hiy, (float)(H - 1));
    if (!(lox <= hix) || !(loy <= hiy)) return;

    d->ok = 1;
    d->r2 = r2;
    d->depth = w;
    d->ex = ex; d->ey = ey;
    d->A00 = A00; d->A01 = A01; d->A11 = A11;
    d->hx = hx; d->hy = hy;
    d->extx = extx; d->exty = exty;
    d->px0 = (int)lox; d->px1 = (int)hix;
    d->py0 = (int)loy; d->py1 = (int)hiy;
    d->p0x = p0x; d->p0y = p0y;
    d->rd2 = rd2;
}

/* x-coordinate of the ellipse boundary on the horizontal line y = ey + dy */
static float chord_x(const disc_t *d, float det, float dy, int right)
{
    const float t1 = d->A01 * dy;
    const float t2 = fmaf(-dy, dy, d->A11);
    const float t3 = sqrtf(fmaxf(det * t2, 0.0f));
    if (OR_PLANT == 5) right = !right;
    return d->ex + (right ? (t1 + t3) : (t1 - t3)) / d->A11;
}

/* Tile-column range [*c0, *c1] touched in tile row ty; returns 0 if none. */
static int row_tiles(const disc_t *d, int mode, int ty, int tw, int th, int *c0, int *c1)
{
    if (mode != OR_EXACT || !(d->A00 > 0.0f && d->A11 > 0.0f)) {
        *c0 = d->px0 / tw;
        *c1 = d->px1 / tw;
        return 1;
    }
    const int r0 = d->py0 > ty * th ? d->py0 : ty * th;
    const int r1 = d->py1 < ty * th + th - 1 ? d->py1 : ty * th + th - 1;
    const float d0 = ((float)r0 + 0.5f) - d->ey;
    const float d1 = ((float)r1 + 0.5f) - d->ey;
    const float det = fmaxf(fmaf(d->A00, d->A11, -(d->A01 * d->A01)), 0.0f);
    const float sl = d->A01 / d->hx; /* dy of the rightmost point; leftmost is -sl */
    float xmin, xmax;
    const float yl = -sl;
    if (yl < d0) xmin = chord_x(d, det, d0, 0);
    else if (yl > d1) xmin = chord_x(d, det, d1, 0);
    else xmin = d->ex - d->hx;
    const float yr = sl;
    if (yr < d0) xmax = chord_x(d, det, d0, 1);
    else if (yr > d1) xmax = chord_x(d, det, d1, 1);
    else xmax = d->ex + d->hx;
    float fl = ceilf(xmin - 0.5f), fh = floorf(xmax - 0.5f);
    fl = fmaxf(fl, (float)d->px0);
    fh = fminf(fh, (float)d->px1);
    int ok = fl <= fh;
    if (d->rd2 >= 0.0f) {
        /* low-pass disc: its chord at the band's row nearest to the centre;
         * the row's columns are the hull of both ranges */
        const float lo = (float)r0 + 0.5f, hi = (float)r1 + 0.5f;
        const float dy = d->p0y < lo ? lo - d->p0y : (d->p0y > hi ? d->p0y - hi : 0.0f);
        const float tt = fmaf(-dy, dy, d->rd2);
        if (tt >= 0.0f) {
            const float h = sqrtf(tt);
            float gl = ceilf((d->p0x - h) - 0.5f), gh = floorf((d->p0x + h) - 0.5f);
            gl = fmaxf(gl, (float)d->px0);
            gh = fminf(gh, (float)d->px1);
            if (gl <= gh) {
                fl = ok ? fminf(fl, gl) : gl;
                fh = ok ? fmaxf(fh, gh) : gh;
                ok = 1;
            }
        }
    }
    if (!ok) return 0;
    *c0 = (int)fl / tw;
    *c1 = (int)fh / tw;
    return 1;
}

static uint32_t disc_count(const disc_t *d, int mode, int tw, int th)
{
    if (!d->ok) return 0;
    uint32_t c = 0;
    for (int ty = d->py0 / th; ty <= d->py1 / th; ty++) {
        int c0, c1;
        if (row_tiles(d, mode, ty, tw, th, &c0, &c1)) c += (uint32_t)(c1 - c0 + 1);
    }
    return c;
}

/* Per-surfel discrete results for one view.
 * out_count[n]: tiles touched; out_depth_bits[n]: float bits of the depth;
 * out_r2[n]; out_rect[4n]: px0,px1,py0,py1 (or -1); out_ell[9n]: ex,ey,A00,A01,A11,hx,hy,extx,exty. */
void or_bin_view(int64_t n, const float *mu, const float *tu, const float *tv, const float *s, const float *o,
                 const float *cam, float chi2, float znear, int oprad, int mode, int lowpass, int tw, int th,
                 uint32_t *out_count, uint32_t *out_depth_bits, float *out_r2, int32_t *out_rect, float *out_ell)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        disc_t d;
        disc_surfel(mu + 3 * i, tu + 3 * i, tv + 3 * i, s[2 * i], s[2 * i + 1], o[i], cam, chi2, znear, oprad, mode, lowpass,
                    &d);
        out_count[i] = disc_count(&d, mode, tw, th);
        out_depth_bits[i] = d.ok ? f_float_to_bits(d.depth) : 0xFFFFFFFFu;
        out_r2[i] = d.ok ? d.r2 : 0.0f;
        if (out_rect) {
            out_rect[4 * i + 0] = d.ok ? d.px0 : -1;
            out_rect[4 * i + 1] = d.ok ? d.px1 : -1;
            out_rect[4 * i + 2] = d.ok ? d.py0 : -1;
            out_rect[4 * i + 3] = d.ok ? d.py1 : -1;
        }
        if (out_ell) {
            float e[9] = {d.ex, d.ey, d.A00, d.A01, d.A11, d.hx, d.hy, d.extx, d.exty};
            memcpy(out_ell + 9 * i, e, sizeof(e));
        }
    }
}

/* Emit (key, value) pairs of one view in surfel order, tiles row-major per surfel.
 * key = (tile_base + ty*tiles_x + tx) << 32 | depth_bits; value = value_base + i.
 * Returns the number of pairs (writes at most cap). */
int64_t or_emit_view(int64_t n, const float *mu, const float *tu, const float *tv, const float *s, const float *o,
                     const float *cam, float chi2, float znear, int oprad, int mode, int lowpass, int tw, int th,
                     uint32_t tile_base, uint32_t value_base, uint64_t *keys, uint32_t *vals, int64_t cap)
{
    const int W = (int)cam[16];
    const int tiles_x = (W + tw - 1) / tw;
    int64_t p = 0;
    for (int64_t i = 0; i < n; i++) {
        disc_t d;
        disc_surfel(mu + 3 * i, tu + 3 * i, tv + 3 * i, s[2 * i], s[2 * i + 1], o[i], cam, chi2, znear, oprad, mode, lowpass,
                    &d);
        if (!d.ok) continue;
        const uint64_t db = f_float_to_bits(d.depth);
        for (int ty = d.py0 / th; ty <= d.py1 / th; ty++) {
            int c0, c1;
            if (!row_tiles(&d, mode, ty, tw, th, &c0, &c1)) continue;
            for (int tx = c0; tx <= c1; tx++) {
                if (p < cap) {
                    keys[p] = ((uint64_t)(tile_base + (uint32_t)(ty * tiles_x + tx)) << 32) | db;
                    vals[p] = value_base + (uint32_t)i;
                }
                p++;
            }
        }
    }
    return p;
}

/* Exposed for the pin that checks it against log(): rho(o) >= 2 ln(255 o). */
float or_rho_opacity(float o) { return rho_opacity(o); }

/* ------------------------------------------------------------------ */
/* (2) value path, float64                                             */
/* ------------------------------------------------------------------ */

#define OR_ALPHA_MIN (1.0 / 255.0)
#define OR_ALPHA_MAX 0.99

typedef struct {
    double xc[3], a[3], b[3]; /* camera-space centre and scaled tangent axes s_u R t_u, s_v R t_v */
} surf64_t;

/* Solve A x = y for 3x3 A (column-major columns c0,c1,c2) by Gaussian
 * elimination with partial pivoting. Returns 0 if singular. */
static int solve3(const double c0[3], const double c1[3], const double c2[3], const double y[3], double x[3])
{
    double m[3][4];
    for (int r = 0; r < 3; r++) { m[r][0] = c0[r]; m[r][1] = c1[r]; m[r][2] = c2[r]; m[r][3] = y[r]; }
    for (int k = 0; k < 3; k++) {
        int piv = k;
        for (int r = k + 1; r < 3; r++) if (fabs(m[r][k]) > fabs(m[piv][k])) piv = r;
        if (m[piv][k] == 0.0) return 0;
        if (piv != k) for (int c = 0; c < 4; c++) { double tmp = m[k][c]; m[k][c] = m[piv][c]; m[piv][c] = tmp; }
        for (int r = k + 1; r < 3; r++) {
            double f = m[r][k] / m[k][k];
            for (int c = k; c < 4; c++) m[r][c] -= f * m[k][c];
        }
    }
    for (int k = 2; k >= 0; k--) {
        double acc = m[k][3];
        for (int c = k + 1; c < 3; c++) acc -= m[k][c] * x[c];
        x[k] = acc / m[k][k];
    }
    return 1;
}

/* Transposed solve: A^T x = y. */
static int solve3T(const double c0[3], const double c1[3], const double c2[3], const double y[3], double x[3])
{
    double r0[3] = {c0[0], c0[1], c0[2]}, r1[3] = {c1[0], c1[1], c1[2]}, r2[3] = {c2[0], c2[1], c2[2]};
    /* A^T has rows c0,c1,c2, i.e. columns (c0[k],c1[k],c2[k]) */
    double k0[3] = {r0[0], r1[0], r2[0]}, k1[3] = {r0[1], r1[1], r2[1]}, k2[3] = {r0[2], r1[2], r2[2]};
    return solve3(k0, k1, k2, y, x);
}

static void prep_surfels(int64_t n, const double *mu, const double *tu, const double *tv, const double *s,
                         const double *cam, surf64_t *out)
{
    const double *R = cam, *t = cam + 9;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < 3; k++) {
            out[i].xc[k] = R[3 * k] * mu[3 * i] + R[3 * k + 1] * mu[3 * i + 1] + R[3 * k + 2] * mu[3 * i + 2] + t[k];
            out[i].a[k] = s[2 * i] * (R[3 * k] * tu[3 * i] + R[3 * k + 1] * tu[3 * i + 1] + R[3 * k + 2] * tu[3 * i + 2]);
            out[i].b[k] = s[2 * i + 1] * (R[3 * k] * tv[3 * i] + R[3 * k + 1] * tv[3 * i + 1] + R[3 * k + 2] * tv[3 * i + 2]);
        }
    }
}

/* Ray through pixel centre vs surfel plane: xc + u a + v b = lam * dir.
 * Returns 1 with (u, v, lam) if the system is regular. */
static int ray_splat(const surf64_t *sf, const double dir[3], double *u, double *v, double *lam)
{
    double c2[3] = {-dir[0], -dir[1], -dir[2]};
    double y[3] = {-sf->xc[0], -sf->xc[1], -sf->xc[2]};
    double x[3];
    if (!solve3(sf->a, sf->b, c2, y, x)) return 0;
    *u = x[0]; *v = x[1]; *lam = x[2];
    return 1;
}

typedef struct { double w; int pos; } wsel_t;

static int cmp_wsel(const void *pa, const void *pb)
{
    const wsel_t *a = (const wsel_t *)pa, *b = (const wsel_t *)pb;
    if (a->w > b->w) return -1;
    if (a->w < b->w) return 1;
    return (a->pos < b->pos) ? -1 : (a->pos > b->pos);
}

typedef struct {
    int idx;       /* position in the canonical order */
    double u, v, lam, G, alpha, T; /* T = transmittance before this surfel */
    int clamped;
    int filt;      /* low-pass term won: rho = 2 (dx^2 + dy^2) */
    double dx, dy; /* pixel centre minus projected centre (low-pass) */
} contrib_t;

typedef struct {
    contrib_t *c;
    int n, cap;
    wsel_t *ws;
    int wcap;
} scratch_t;

static void push_contrib(scratch_t *s, const contrib_t *c)
{
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 256;
        s->c = (contrib_t *)realloc(s->c, (size_t)s->cap * sizeof(contrib_t));
    }
    s->c[s->n++] = *c;
}

/* Front-to-back walk for one pixel. Fills s->c with the composited surfels,
 * returns final T. diag (may be NULL) receives threshold distances. */
static double walk_pixel(const surf64_t *sf, const double *o, const int *order, int n_order, const double *r2,
                         const double *cam, int px, int py, double t_eps, int lowpass, scratch_t *s, double *diag)
{
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const double dir[3] = {((double)px + 0.5 - cx) / fx, ((double)py + 0.5 - cy) / fy, 1.0};
    double T = 1.0;
    double dmin_r = INFINITY, dmin_a = INFINITY, dmin_t = INFINITY, cond = 0.0, cond1 = 0.0;
    s->n = 0;
    for (int k = 0; k < n_order; k++) {
        const int i = order[k];
        double u = 0.0, v = 0.0, lam = 0.0;
        const int hit = ray_splat(&sf[i], dir, &u, &v, &lam) && lam > 0.0;
        if (!hit && !lowpass) continue;
        double d2 = hit ? u * u + v * v : INFINITY; /* rho of the surfel's own Gaussian */
        double ddx = 0.0, ddy = 0.0;
        int filt = 0;
        if (lowpass) {
            /* screen-space term: pixel distance to the projected centre */
            const double *xc = sf[i].xc;
            ddx = ((double)px + 0.5) - (fx * xc[0] / xc[2] + cx);
            ddy = ((double)py + 0.5) - (fy * xc[1] / xc[2] + cy);
            const double rho2 = ((OR_PLANT == 6) ? 1.0 : 2.0) * (ddx * ddx + ddy * ddy);
            const double rho3 = d2 <= r2[i] ? d2 : INFINITY;
            if (diag && o[i] * exp(-0.5 * r2[i]) >= OR_ALPHA_MIN * 0.5) {
                double rel = fabs(fmin(d2, rho2) - r2[i]) / r2[i];
                if (rel < dmin_r) dmin_r = rel;
            }
            filt = rho2 < rho3;
            d2 = filt ? rho2 : rho3;
        } else if (diag && o[i] * exp(-0.5 * r2[i]) >= OR_ALPHA_MIN * 0.5) {
            double rel = fabs(d2 - r2[i]) / r2[i];
            if (rel < dmin_r) dmin_r = rel;
        }
        if (!(d2 <= r2[i])) continue;
        const double G = (OR_PLANT == 1) ? exp(-d2) : exp(-0.5 * d2);
        double a = o[i] * G;
        int clamped = 0;
        if (a > OR_ALPHA_MAX) { a = OR_ALPHA_MAX; clamped = 1; }
        if (diag) {
            double rel = fabs(a - OR_ALPHA_MIN) / OR_ALPHA_MIN;
            if (rel < dmin_a) dmin_a = rel;
        }
        if (a < OR_ALPHA_MIN) continue;
        const double Tn = T * (1.0 - a);
        contrib_t c = {k, u, v, lam, G, a, (OR_PLANT == 2) ? Tn : T, clamped, filt, ddx, ddy};
        push_contrib(s, &c);
        if (diag && filt) {
            /* d rho / d pixel = 4 (dx, dy) */
            const double sens = clamped ? 0.0 : 0.5 * a * 4.0 * sqrt(ddx * ddx + ddy * ddy);
            cond += sens * T;
            if (sens > cond1) cond1 = sens;
        } else if (diag) {
            /* sensitivity of d2 to the pixel position: d(u,v,lam)/dx = B^-1 lam e_x / fx */
            double c2[3] = {-dir[0], -dir[1], -dir[2]};
            double ex_[3] = {lam / fx, 0.0, 0.0}, ey_[3] = {0.0, lam / fy, 0.0}, zx[3], zy[3];
            if (solve3(sf[i].a, sf[i].b, c2, ex_, zx) && solve3(sf[i].a, sf[i].b, c2, ey_, zy)) {
                const double gx = 2.0 * (u * zx[0] + v * zx[1]);
                const double gy = 2.0 * (u * zy[0] + v * zy[1]);
                const double gn = sqrt(gx * gx + gy * gy);
                const double sens = clamped ? 0.0 : 0.5 * a * gn;
                cond += sens * T;
                if (sens > cond1) cond1 = sens;
            }
        }
        if (diag) {
            double rel = fabs(Tn - t_eps) / t_eps;
            if (rel < dmin_t) dmin_t = rel;
        }
        T = Tn;
        if (T < t_eps) break;
    }
    if (diag) { diag[0] = dmin_r; diag[1] = dmin_a; diag[2] = dmin_t; diag[4] = cond; diag[5] = cond1; }
    return T;
}

/* Contributors of one pixel in front-to-back order: surfel id, u, v, alpha, T
 * before it, selection flag. Returns the count (writes at most cap). */
int or_pixel_walk(int64_t n, const double *mu, const double *tu, const double *tv, const double *s, const double *o,
                  const int *order, int n_order, const double *r2, const double *cam, int px, int py, int K,
                  double t_eps, int lowpass, int32_t *out_id, double *out_uvat, uint8_t *out_sel, int cap);

/* Select Top-K contributors: sets sel[j]=1 for chosen entries of s->c. Returns
 * the gap omega_(K) - omega_(K+1) (INFINITY if no (K+1)-th). K <= 0: all. */
static double select_topk(scratch_t *s, int K, unsigned char *sel)
{
    const int n = s->n;
    if (K <= 0 || n <= K) {
        for (int j = 0; j < n; j++) sel[j] = 1;
        return INFINITY;
    }
    if (s->wcap < n) {
        s->wcap = n;
        s->ws = (wsel_t *)realloc(s->ws, (size_t)n * sizeof(wsel_t));
    }
    for (int j = 0; j < n; j++) { s->ws[j].w = s->c[j].alpha * s->c[j].T; s->ws[j].pos = j; sel[j] = 0; }
    qsort(s->ws, (size_t)n, sizeof(wsel_t), cmp_wsel);
    for (int j = 0; j < K; j++) sel[s->ws[(OR_PLANT == 3) ? n - 1 - j : j].pos] = 1;
    return s->ws[K - 1].w - s->ws[K].w;
}

/* Forward render of a list of pixels.
 *  order[n_order]: canonical order (non-culled surfels sorted by (float depth bits, id)).
 *  r2[n]: per-surfel support radius^2 from the discrete path.
 *  feat[n*D] (or NULL), K (<=0: dense).
 * Outputs per pixel: rgb[3], T, F[D] (if feat), topk[K] surfel ids (ascending list
 * order, -1 padded; if K>0), ncontrib, sumw, diag[6], hash (contributor ids + selection). */
void or_render(int64_t n, const double *mu, const double *tu, const double *tv, const double *s, const double *o,
               const double *rgb, const double *feat, int D, const int *order, int n_order, const double *r2,
               const double *cam, int64_t npix, const int32_t *pix, int K, double t_eps, int lowpass,
               double *out_rgb, double *out_T, double *out_F, int32_t *out_topk, int32_t *out_ncontrib,
               double *out_sumw, double *out_diag, uint64_t *out_hash)
{
    surf64_t *sf = (surf64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(surf64_t));
    prep_surfels(n, mu, tu, tv, s, cam, sf);
#pragma omp parallel
    {
        scratch_t sc = {0};
        unsigned char *sel = NULL;
        int selcap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < npix; p++) {
            double diag[6] = {0};
            const double T = walk_pixel(sf, o, order, n_order, r2, cam, pix[2 * p], pix[2 * p + 1], t_eps, lowpass, &sc, diag);
            if (selcap < sc.n) { selcap = sc.n; sel = (unsigned char *)realloc(sel, (size_t)selcap); }
            diag[3] = select_topk(&sc, K, sel);
            double c3[3] = {0, 0, 0}, sw = 0.0;
            uint64_t h = 1469598103934665603ull;
            for (int j = 0; j < sc.n; j++) {
                const int i = order[sc.c[j].idx];
                const double w = sc.c[j].alpha * sc.c[j].T;
                for (int c = 0; c < 3; c++) c3[c] += w * rgb[3 * i + c];
                sw += w;
                h = (h ^ (uint64_t)(i * 4 + sel[j] * 2 + sc.c[j].filt)) * 1099511628211ull;
            }
            for (int c = 0; c < 3; c++) out_rgb[3 * p + c] = c3[c];
            out_T[p] = T;
            if (out_sumw) out_sumw[p] = sw;
            if (out_ncontrib) out_ncontrib[p] = sc.n;
            if (out_hash) out_hash[p] = h;
            if (out_diag) memcpy(out_diag + 6 * p, diag, sizeof(diag));
            if (feat && out_F) {
                double *F = out_F + (size_t)p * D;
                for (int c = 0; c < D; c++) F[c] = 0.0;
                for (int j = 0; j < sc.n; j++) {
                    if (!sel[j]) continue;
                    const int i = order[sc.c[j].idx];
                    const double w = sc.c[j].alpha * sc.c[j].T;
                    for (int c = 0; c < D; c++) F[c] += w * feat[(size_t)i * D + c];
                }
            }
            if (out_topk && K > 0) {
                int m = 0;
                for (int j = 0; j < sc.n && m < K; j++) if (sel[j]) out_topk[p * K + m++] = order[sc.c[j].idx];
                for (; m < K; m++) out_topk[p * K + m] = -1;
            }
        }
        free(sc.c); free(sc.ws); free(sel);
    }
    free(sf);
}

/* Gradient of L = sum_p [gC.C + gF.F + gT*T] with respect to surfel parameters.
 * Outputs (accumulated, caller zeroes): g_mu[3n], g_tu[3n], g_tv[3n], g_s[2n],
 * g_o[n], g_rgb[3n], g_feat[n*D] (if feat). gF, gT may be NULL. */
void or_render_grad(int64_t n, const double *mu, const double *tu, const double *tv, const double *s, const double *o,
                    const double *rgb, const double *feat, int D, const int *order, int n_order, const double *r2,
                    const double *cam, int64_t npix, const int32_t *pix, int K, double t_eps, int lowpass,
                    const double *gC, const double *gF, const double *gT,
                    double *g_mu, double *g_tu, double *g_tv, double *g_s, double *g_o, double *g_rgb, double *g_feat)
{
    const double *R = cam;
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    surf64_t *sf = (surf64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(surf64_t));
    prep_surfels(n, mu, tu, tv, s, cam, sf);
#pragma omp parallel
    {
        scratch_t sc = {0};
        unsigned char *sel = NULL;
        int selcap = 0;
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < npix; p++) {
            const int px = pix[2 * p], py = pix[2 * p + 1];
            const double Tf = walk_pixel(sf, o, order, n_order, r2, cam, px, py, t_eps, lowpass, &sc, NULL);
            if (selcap < sc.n) { selcap = sc.n; sel = (unsigned char *)realloc(sel, (size_t)selcap); }
            select_topk(&sc, K, sel);
            const double dir[3] = {((double)px + 0.5 - cx) / fx, ((double)py + 0.5 - cy) / fy, 1.0};
            const double *gc = gC + 3 * p;
            const double *gf = gF ? gF + (size_t)p * D : NULL;
            const double gt = gT ? gT[p] : 0.0;
            /* back to front: suffix = sum_{k>j} omega_k s_k + T_final * gT */
            double suffix = Tf * gt;
            for (int j = sc.n - 1; j >= 0; j--) {
                const contrib_t *c = &sc.c[j];
                const int i = order[c->idx];
                const double w = c->alpha * c->T;
                double sj = gc[0] * rgb[3 * i] + gc[1] * rgb[3 * i + 1] + gc[2] * rgb[3 * i + 2];
                if (gf && sel[j]) {
                    double acc = 0.0;
                    for (int ch = 0; ch < D; ch++) acc += gf[ch] * feat[(size_t)i * D + ch];
                    sj += acc;
                }
                const double dL_da = c->T * sj - suffix / (1.0 - c->alpha);
                suffix += w * sj;
                for (int ch = 0; ch < 3; ch++) {
#pragma omp atomic
                    g_rgb[3 * i + ch] += w * gc[ch];
                }
                if (gf && sel[j] && g_feat) {
                    for (int ch = 0; ch < D; ch++) {
#pragma omp atomic
                        g_feat[(size_t)i * D + ch] += w * gf[ch];
                    }
                }
                if (c->clamped) continue; /* alpha held at 0.99: no dependence on o, u, v */
                /* alpha = o G, G = exp(-rho/2) */
#pragma omp atomic
                g_o[i] += dL_da * c->G;
                if (c->filt) {
                    /* rho = 2 |x - p|^2 with p = (fx X/Z + cx, fy Y/Z + cy), (X, Y, Z) = R mu + t:
                     * dL/dp = dL/drho * (-4 (dx, dy)), dL/drho = -dL/dalpha alpha / 2 */
                    const double grho = -0.5 * dL_da * c->alpha;
                    const double sgn = (OR_PLANT == 7) ? -1.0 : 1.0;
                    const double gpx = sgn * grho * (-4.0 * c->dx), gpy = sgn * grho * (-4.0 * c->dy);
                    const double *xc = sf[i].xc;
                    const double gxc[3] = {gpx * fx / xc[2], gpy * fy / xc[2],
                                           -(gpx * fx * xc[0] + gpy * fy * xc[1]) / (xc[2] * xc[2])};
                    for (int k = 0; k < 3; k++) {
#pragma omp atomic
                        g_mu[3 * i + k] += R[k] * gxc[0] + R[3 + k] * gxc[1] + R[6 + k] * gxc[2];
                    }
                    continue;
                }
                const double gu = dL_da * (-c->alpha * c->u);
                const double gv = dL_da * (-c->alpha * c->v);
                /* implicit differentiation of B (u,v,lam) = -xc, B = [a | b | -dir]:
                 * d(u,v,lam) = -B^-1 (dxc + dB (u,v,lam)); dL = -y . (dxc + dB s), y = B^-T (gu,gv,0) */
                const double c2[3] = {-dir[0], -dir[1], -dir[2]};
                const double g3[3] = {gu, gv, 0.0};
                double y[3];
                if (!solve3T(sf[i].a, sf[i].b, c2, g3, y)) continue;
                /* dxc/dmu = R; dB s / d(tu) = u * s_u * R; d/d(s_u) = u * (R tu) */
                double Rty[3];
                for (int k = 0; k < 3; k++) Rty[k] = R[k] * y[0] + R[3 + k] * y[1] + R[6 + k] * y[2];
                const double su_ = s[2 * i], sv_ = s[2 * i + 1];
                /* (R tu) . y = tu . (R^T y) */
                double tuy = 0.0, tvy = 0.0;
                for (int k = 0; k < 3; k++) { tuy += tu[3 * i + k] * Rty[k]; tvy += tv[3 * i + k] * Rty[k]; }
                for (int k = 0; k < 3; k++) {
#pragma omp atomic
                    g_mu[3 * i + k] += (OR_PLANT == 4) ? Rty[k] : -Rty[k];
#pragma omp atomic
                    g_tu[3 * i + k] += -c->u * su_ * Rty[k];
#pragma omp atomic
                    g_tv[3 * i + k] += -c->v * sv_ * Rty[k];
                }
                /* a = s_u R tu, so (d a / d s_u) . y = (R tu) . y */
#pragma omp atomic
                g_s[2 * i] += -c->u * tuy;
#pragma omp atomic
                g_s[2 * i + 1] += -c->v * tvy;
            }
        }
        free(sc.c); free(sc.ws); free(sel);
    }
    free(sf);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_pixel_walk(int64_t n, const double *mu, const double *tu, const double *tv, const double *s, const double *o,
                  const int *order, int n_order, const double *r2, const double *cam, int px, int py, int K,
                  double t_eps, int lowpass, int32_t *out_id, double *out_uvat, uint8_t *out_sel, int cap)
{
    surf64_t *sf = (surf64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(surf64_t));
    prep_surfels(n, mu, tu, tv, s, cam, sf);
    scratch_t sc = {0};
    walk_pixel(sf, o, order, n_order, r2, cam, px, py, t_eps, lowpass, &sc, NULL);
    unsigned char *sel = (unsigned char *)malloc((size_t)(sc.n > 0 ? sc.n : 1));
    select_topk(&sc, K, sel);
    for (int j = 0; j < sc.n && j < cap; j++) {
        out_id[j] = order[sc.c[j].idx];
        out_uvat[4 * j + 0] = sc.c[j].u;
        out_uvat[4 * j + 1] = sc.c[j].v;
        out_uvat[4 * j + 2] = sc.c[j].alpha;
        out_uvat[4 * j + 3] = sc.c[j].T;
        out_sel[j] = sel[j];
    }
    const int cnt = sc.n;
    free(sc.c); free(sc.ws); free(sel); free(sf);
    return cnt;
}
