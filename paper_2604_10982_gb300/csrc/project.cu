// a1: per (view, surfel) projection, culling, ray-splat setup and binning bounds.
//
// The surfel plane P(u,v) = mu + s_u u t_u + s_v v t_v (Sec. 3.1) maps to
// pixel-homogeneous coordinates through the 3x3 matrix
//     M = [ K R (s_u t_u) | K R (s_v t_v) | K (R mu + t) ],  p_h = M (u, v, 1)^T,
// so the ray through a pixel meets the plane at (u, v, 1) ~ M^-1 p_h: the
// 2D-surfel ray-splat intersection written as one linear map. The kernel
// stores adj(M') for the renderer (M' = M shifted so the projected centre is
// the pixel origin, which keeps the float32 arithmetic well conditioned) and
// the bounds of the projected support ellipse for binning. The ellipse comes
// from the dual conic C* = M diag(r^2, r^2, -1) M^T: centre C*_13 / C*_33 and
// shape Sigma_ij = (C*_i3 C*_j3 - C*_ij C*_33) / C*_33^2, whose diagonal gives
// the half-widths sqrt(chi^2 Sigma'_11), sqrt(chi^2 Sigma'_22) of Sec. 5
// (Precise Tile Intersection) exactly under perspective.
#include "discrete.cuh"

namespace psi {

void fill_frame_params(FrameParams &fp, const psi_camera *cams, int n_views, const psi_render_opts *o, int64_t n)
{
    fp.n_views = n_views;
    fp.mode = o->mode;
    fp.n = n;
    fp.tile_w = o->tile_w;
    fp.tile_h = o->tile_h;
    fp.chi2 = o->chi2;
    fp.z_near = o->z_near;
    fp.t_eps = o->t_eps;
    fp.opacity_radius = o->opacity_radius;
    fp.top_k = o->top_k;
    fp.lowpass = o->lowpass;
    uint32_t tb = 0;
    int64_t pb = 0;
    for (int v = 0; v < n_views; ++v) {
        ViewParams &vp = fp.v[v];
        for (int k = 0; k < 9; ++k) vp.R[k] = cams[v].R[k];
        for (int k = 0; k < 3; ++k) vp.t[k] = cams[v].t[k];
        vp.fx = cams[v].fx;
        vp.fy = cams[v].fy;
        vp.cx = cams[v].cx;
        vp.cy = cams[v].cy;
        vp.W = cams[v].width;
        vp.H = cams[v].height;
        vp.tiles_x = (vp.W + o->tile_w - 1) / o->tile_w;
        vp.tiles_y = (vp.H + o->tile_h - 1) / o->tile_h;
        vp.tile_base = tb;
        vp.pad = 0;
        vp.pix_base = pb;
        tb += static_cast<uint32_t>(vp.tiles_x * vp.tiles_y);
        pb += static_cast<int64_t>(vp.W) * vp.H;
    }
    fp.n_tiles_total = tb;
    fp.n_pix_total = pb;
}

namespace {

using namespace disc;

__global__ void __launch_bounds__(256) project_kernel(const __grid_constant__ FrameParams fp, psi_surfels s,
                                                      float4 *__restrict__ records, float4 *__restrict__ bins,
                                                      uint32_t *__restrict__ counts)
{
    const int64_t total = fp.n * fp.n_views;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= total) return;
    const int v = static_cast<int>(r / fp.n);
    const int64_t i = r - static_cast<int64_t>(v) * fp.n;
    const ViewParams &cam = fp.v[v];
    const float *R = cam.R;

    const float m0 = s.mu[3 * i], m1 = s.mu[3 * i + 1], m2 = s.mu[3 * i + 2];
    const float u0 = s.tu[3 * i], u1 = s.tu[3 * i + 1], u2 = s.tu[3 * i + 2];
    const float v0 = s.tv[3 * i], v1 = s.tv[3 * i + 1], v2 = s.tv[3 * i + 2];
    const float su = s.scale[2 * i], sv = s.scale[2 * i + 1];
    const float o = s.opacity[i];

    // camera-space centre and scaled tangent axes (explicit FMA chains)
    float xc[3], uu[3], vv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        xc[k] = fma(R[3 * k + 2], m2, fma(R[3 * k + 1], m1, fma(R[3 * k], m0, cam.t[k])));
        const float au = fma(R[3 * k + 2], u2, fma(R[3 * k + 1], u1, mul(R[3 * k], u0)));
        const float av = fma(R[3 * k + 2], v2, fma(R[3 * k + 1], v1, mul(R[3 * k], v0)));
        uu[k] = mul(su, au);
        vv[k] = mul(sv, av);
    }
    if (!(o >= kAlphaMin)) {
        counts[r] = 0;
        return;
    }
    float r2 = fp.chi2;
    if (fp.opacity_radius) r2 = fminf(fp.chi2, opacity_radius2(o));
    const float r2b = mul(r2, kBinInflate);

    // the whole binning disc must lie beyond the near plane
    const float w = xc[2];
    const float nab = sqrt(fma(uu[2], uu[2], mul(vv[2], vv[2])));
    const float rb = sqrt(r2b);
    const float zmin = fma(-rb, nab, w);
    if (!(zmin > fp.z_near)) {
        counts[r] = 0;
        return;
    }

    // shifted pixel-homogeneous columns of M'
    const float fx = cam.fx, fy = cam.fy, cx = cam.cx, cy = cam.cy;
    const float mcx = fma(fx, xc[0], mul(cx, xc[2]));
    const float mcy = fma(fy, xc[1], mul(cy, xc[2]));
    const float p0x = div(mcx, w), p0y = div(mcy, w);
    float mu_[3], mv_[3], mc_[3];
    mu_[0] = fma(-p0x, uu[2], fma(fx, uu[0], mul(cx, uu[2])));
    mu_[1] = fma(-p0y, uu[2], fma(fy, uu[1], mul(cy, uu[2])));
    mu_[2] = uu[2];
    mv_[0] = fma(-p0x, vv[2], fma(fx, vv[0], mul(cx, vv[2])));
    mv_[1] = fma(-p0y, vv[2], fma(fy, vv[1], mul(cy, vv[2])));
    mv_[2] = vv[2];
    mc_[0] = fma(-p0x, w, mcx);
    mc_[1] = fma(-p0y, w, mcy);
    mc_[2] = w;

    // dual conic of the binning disc
    auto conic = [&](int a, int b) { return fma(r2b, fma(mu_[a], mu_[b], mul(mv_[a], mv_[b])), -mul(mc_[a], mc_[b])); };
    const float C00 = conic(0, 0), C01 = conic(0, 1), C02 = conic(0, 2);
    const float C11 = conic(1, 1), C12 = conic(1, 2), C22 = conic(2, 2);
    if (!(C22 < 0.0f)) {
        counts[r] = 0;
        return;
    }
    Bin b;
    b.ex = add(p0x, div(C02, C22));
    b.ey = add(p0y, div(C12, C22));
    const float q = mul(C22, C22);
    b.A00 = div(fma(C02, C02, -mul(C00, C22)), q);
    b.A11 = div(fma(C12, C12, -mul(C11, C22)), q);
    b.A01 = div(fma(C02, C12, -mul(C01, C22)), q);
    const float hx = sqrt(fmaxf(b.A00, 0.0f));
    const float hy = sqrt(fmaxf(b.A11, 0.0f));
    float extx = hx, exty = hy;
    if (fp.mode == PSI_ISECT_SPHERE) {
        const float mid = mul(0.5f, add(b.A00, b.A11));
        const float dd = mul(0.5f, sub(b.A00, b.A11));
        const float lam = add(mid, sqrt(fma(dd, dd, mul(b.A01, b.A01))));
        float Rs = sqrt(fmaxf(lam, 0.0f));
        Rs = fmaxf(Rs, fmaxf(hx, hy));
        extx = Rs;
        exty = Rs;
    }
    if (!(fabsf(b.ex) <= kFltMax && fabsf(b.ey) <= kFltMax && extx <= kFltMax && exty <= kFltMax)) {
        counts[r] = 0;
        return;
    }
    float lox = ceilf(sub(sub(b.ex, extx), 0.5f)), hix = floorf(sub(add(b.ex, extx), 0.5f));
    float loy = ceilf(sub(sub(b.ey, exty), 0.5f)), hiy = floorf(sub(add(b.ey, exty), 0.5f));
    // low-pass filter: the rectangle also covers the disc 2 |x - p0|^2 <= r2b
    const bool lp = fp.lowpass != 0;
    b.p0x = p0x;
    b.p0y = p0y;
    b.rd2 = lp ? mul(r2b, 0.5f) : -1.0f;
    if (lp) {
        const float rd = sqrt(b.rd2);
        lox = fminf(lox, ceilf(sub(sub(p0x, rd), 0.5f)));
        hix = fmaxf(hix, floorf(sub(add(p0x, rd), 0.5f)));
        loy = fminf(loy, ceilf(sub(sub(p0y, rd), 0.5f)));
        hiy = fmaxf(hiy, floorf(sub(add(p0y, rd), 0.5f)));
    }
    lox = fmaxf(lox, 0.0f);
    loy = fmaxf(loy, 0.0f);
    hix = fminf(hix, static_cast<float>(cam.W - 1));
    hiy = fminf(hiy, static_cast<float>(cam.H - 1));
    if (!(lox <= hix) || !(loy <= hiy)) {
        counts[r] = 0;
        return;
    }
    b.px0 = static_cast<int>(lox);
    b.px1 = static_cast<int>(hix);
    b.py0 = static_cast<int>(loy);
    b.py1 = static_cast<int>(hiy);
    counts[r] = count_tiles(b, fp.mode, fp.tile_w, fp.tile_h);
    store_bin(bins + bin_stride(lp) * r, b, w, lp);

    // render record (80 bytes): rows of adj(M') (q = adj(M') (x - p0x, y - p0y, 1)),
    // projected centre, opacity, support radius^2, colour, covered-pixel rectangle
    const float a00 = mv_[1] * mc_[2] - mv_[2] * mc_[1];
    const float a01 = mv_[2] * mc_[0] - mv_[0] * mc_[2];
    const float a02 = mv_[0] * mc_[1] - mv_[1] * mc_[0];
    const float a10 = mc_[1] * mu_[2] - mc_[2] * mu_[1];
    const float a11 = mc_[2] * mu_[0] - mc_[0] * mu_[2];
    const float a12 = mc_[0] * mu_[1] - mc_[1] * mu_[0];
    const float a20 = mu_[1] * mv_[2] - mu_[2] * mv_[1];
    const float a21 = mu_[2] * mv_[0] - mu_[0] * mv_[2];
    const float a22 = mu_[0] * mv_[1] - mu_[1] * mv_[0];
    float4 *rec = records + 5 * r;
    rec[0] = make_float4(a00, a01, a02, a10);
    rec[1] = make_float4(a11, a12, a20, a21);
    rec[2] = make_float4(a22, p0x, p0y, o);
    rec[3] = make_float4(r2, s.rgb[3 * i], s.rgb[3 * i + 1], s.rgb[3 * i + 2]);
    // rectangle of pixel indices whose centres the binning ellipse may cover
    // (the one the tile lists come from): lets each warp skip whole records
    rec[4] = make_float4(__uint_as_float(static_cast<uint32_t>(b.px0) | (static_cast<uint32_t>(b.px1) << 16)),
                         __uint_as_float(static_cast<uint32_t>(b.py0) | (static_cast<uint32_t>(b.py1) << 16)), 0.0f,
                         0.0f);
}

} // namespace

cudaError_t launch_project(const FrameParams &fp, const psi_surfels &s, float4 *records, float4 *bin_records,
                           uint32_t *tiles_touched, cudaStream_t st)
{
    const int64_t total = fp.n * fp.n_views;
    if (total == 0) return cudaSuccess;
    const int64_t blocks = (total + 255) / 256;
    project_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(fp, s, records, bin_records, tiles_touched);
    return cudaGetLastError();
}

} // namespace psi
