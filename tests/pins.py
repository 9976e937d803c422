"""Pins of the CPU oracle: checks against closed forms, invariants, brute force
and finite differences. Each check raises AssertionError on failure, so the
planted-mistake test can run the same checks against deliberately wrong
oracle builds and expect them to fail.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg


def _cam_f64(cam):
    a = cam.as_array().astype(np.float64)
    return a[:9].reshape(3, 3), a[9:12], a[12], a[13], a[14], a[15]


def fronto_surfel(cam, X, Y, z0, su, sv, o, rgb=(1.0, 1.0, 1.0)):
    """A surfel whose tangent axes are the camera's x and y axes, centred at
    camera-space (X, Y, z0). Returns Surfels (float32) and the exact float32
    camera-space centre as float64."""
    R, t, *_ = _cam_f64(cam)
    xc = np.array([X, Y, z0])
    mu = R.T @ (xc - t)
    s = sg.Surfels(np.array([mu], np.float32), np.array([R[0]], np.float32), np.array([R[1]], np.float32),
                   np.array([[su, sv]], np.float32), np.array([o], np.float32), np.array([rgb], np.float32))
    xc32 = R @ s.mu[0].astype(np.float64) + t
    return s, xc32


def closed_form_alpha(cam, xc, su, sv, o, px, py):
    """alpha at pixel centres for a camera-facing surfel (exact closed form)."""
    _, _, fx, fy, cx, cy = _cam_f64(cam)
    su, sv, o = float(np.float32(su)), float(np.float32(sv)), float(np.float32(o))
    X, Y, z0 = xc
    u = ((px + 0.5 - cx) * z0 / fx - X) / su
    v = ((py + 0.5 - cy) * z0 / fy - Y) / sv
    d2 = u * u + v * v
    return o * np.exp(-0.5 * d2), d2


def concat(*ss):
    return sg.Surfels(*(np.concatenate([getattr(s, f) for s in ss]) for f in
                        ("mu", "tu", "tv", "scale", "opacity", "rgb")))


CAM = sg.look_camera((0.0, -6.0, 1.5), 0.0, 128, 128, 110.0)


def pin_fronto_parallel():
    """A camera-facing surfel reproduces the analytic 2D Gaussian (Sec. 3.1)."""
    s, xc = fronto_surfel(CAM, 0.21, -0.13, 3.0, 0.35, 0.22, 0.8, rgb=(1.0, 0.5, 0.25))
    opts = orc.Opts(mode=orc.EXACT, chi2=9.0)
    out = orc.render(s, CAM, opts)
    pix = out["pixels"]
    a, d2 = closed_form_alpha(CAM, xc, 0.35, 0.22, 0.8, pix[:, 0].astype(float), pix[:, 1].astype(float))
    inside = (d2 <= 9.0) & (a >= 1 / 255)
    safe = (np.abs(d2 - 9.0) > 1e-9) & (np.abs(a - 1 / 255) > 1e-12)
    exp_a = np.where(inside, np.minimum(a, 0.99), 0.0)
    m = safe
    assert m.sum() > 500
    assert np.max(np.abs(out["rgb"][m, 0] - exp_a[m])) < 1e-12
    assert np.max(np.abs(out["rgb"][m, 2] - 0.25 * exp_a[m])) < 1e-12
    assert np.max(np.abs(out["T"][m] - (1.0 - exp_a[m]))) < 1e-12


def _screen_term(cam, s, o, pix, r2):
    """The screen-space term of the 2DGS low-pass filter for one surfel: a
    Gaussian of standard deviation sqrt(2)/2 pixel about the projected centre
    c = K (R mu + t) (dehomogenised), i.e. o exp(-|x - c|^2) with the opacity
    clamp and cut-offs of Sec. 3.1; 0 outside 2 |x - c|^2 <= r2. Also returns
    the squared-distance argument 2 |x - c|^2."""
    R, t, fx, fy, cx, cy = _cam_f64(cam)
    K = np.array([[fx, 0.0, cx], [0.0, fy, cy], [0.0, 0.0, 1.0]])
    h = K @ (R @ s.mu[0].astype(np.float64) + t)
    d = pix.astype(np.float64) + 0.5 - h[:2] / h[2]
    rho = 2.0 * np.sum(d * d, axis=1)
    a = min(float(np.float32(o)), 1.0) * np.exp(-0.5 * rho)
    return np.where((rho <= r2) & (a >= 1 / 255), np.minimum(a, 0.99), 0.0), rho, a


def _edge_on_surfel(cam, xc, su, sv, o):
    """A surfel whose plane contains the camera centre (seen exactly edge on):
    t_u = camera x axis, t_v = unit vector from the camera to the centre."""
    R, t, *_ = _cam_f64(cam)
    xc = np.asarray(xc, np.float64)
    mu = R.T @ (xc - t)
    tu = R.T @ np.array([1.0, 0.0, 0.0])
    tv = R.T @ (xc / np.linalg.norm(xc))
    tv -= tu * (tu @ tv)
    tv /= np.linalg.norm(tv)
    return sg.Surfels(np.array([mu], np.float32), np.array([tu], np.float32), np.array([tv], np.float32),
                      np.array([[su, sv]], np.float32), np.array([o], np.float32), np.array([[1.0, 1.0, 1.0]], np.float32))


def pin_lowpass():
    """2DGS object-space low-pass filter: for one surfel the filtered alpha is
    the larger of the surfel's own alpha (the unfiltered render, pinned above)
    and the screen-space Gaussian term; an edge-on surfel is invisible without
    the filter and exactly the screen-space term with it; a surfel several
    pixels wide is unchanged."""
    cases = [
        fronto_surfel(CAM, 0.10, -0.05, 3.0, 0.01, 0.012, 0.8)[0],   # ~0.4 px: the screen term wins
        fronto_surfel(CAM, -0.2, 0.07, 3.0, 0.10, 0.008, 0.7)[0],    # 3.7 x 0.3 px: both terms win somewhere
        _edge_on_surfel(CAM, (0.13, -0.08, 2.5), 0.3, 0.2, 0.9),
    ]
    rng = np.random.default_rng(8)
    for _ in range(3):  # small surfels at random tilts
        mu = np.array([rng.uniform(-0.4, 0.4), rng.uniform(-0.3, 0.3), rng.uniform(2.0, 4.0)])
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        a = np.cross(n, [0.3, 0.5, 0.8]); a /= np.linalg.norm(a)
        R, t, *_ = _cam_f64(CAM)
        cases.append(sg.Surfels(np.array([R.T @ (mu - t)], np.float32), np.array([R.T @ a], np.float32),
                                np.array([R.T @ np.cross(n, a)], np.float32),
                                np.array(rng.uniform(0.005, 0.03, (1, 2)), np.float32), np.array([0.85], np.float32),
                                np.array([[1.0, 1.0, 1.0]], np.float32)))
    for k, s in enumerate(cases):
        plain = orc.render(s, CAM, orc.Opts(mode=orc.EXACT))
        filt = orc.render(s, CAM, orc.Opts(mode=orc.EXACT, lowpass=True))
        pix = filt["pixels"]
        r2 = float(orc.bin_view(s, CAM, orc.Opts(mode=orc.EXACT, lowpass=True))["r2"][0])
        scr, rho, a_raw = _screen_term(CAM, s, s.opacity[0], pix, r2)
        safe = (np.abs(rho - r2) > 1e-9) & (np.abs(a_raw - 1 / 255) > 1e-12)
        want = np.maximum(1.0 - plain["T"], scr)
        got = 1.0 - filt["T"]
        assert np.max(np.abs(got[safe] - want[safe])) < 1e-12, k
        assert (scr > 0).sum() >= 3, k
        if k == 2:
            assert np.all(plain["T"] == 1.0)
    # several pixels wide: the surfel's own term wins everywhere
    s, _ = fronto_surfel(CAM, 0.21, -0.13, 3.0, 0.35, 0.22, 0.8)
    a = orc.render(s, CAM, orc.Opts(mode=orc.EXACT))
    b = orc.render(s, CAM, orc.Opts(mode=orc.EXACT, lowpass=True))
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["rgb"], b["rgb"])


def pin_rotated_point():
    """A point placed on a tilted surfel at (u0, v0) and projected by hand onto a
    pixel centre is recovered by the ray-splat intersection."""
    rng = np.random.default_rng(3)
    for trial in range(20):
        mu = np.array([rng.uniform(-1, 1), rng.uniform(-2, 2), rng.uniform(0.5, 2.5)])
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        a = np.cross(n, [0.3, 0.5, 0.8]); a /= np.linalg.norm(a)
        b = np.cross(n, a)
        su, sv = rng.uniform(0.1, 0.5, 2)
        s = sg.Surfels(np.array([mu], np.float32), np.array([a], np.float32), np.array([b], np.float32),
                       np.array([[su, sv]], np.float32), np.array([0.9], np.float32), np.array([[1, 1, 1]], np.float32))
        mu64, a64, b64 = (getattr(s, f)[0].astype(np.float64) for f in ("mu", "tu", "tv"))
        su64, sv64 = s.scale[0].astype(np.float64)
        u0, v0 = rng.uniform(-1.2, 1.2, 2)
        P = mu64 + su64 * u0 * a64 + sv64 * v0 * b64
        cam = sg.look_camera((0.0, -6.0, 1.5), 0.0, 128, 128, 110.0)
        R, t, fx, fy, cx, cy = _cam_f64(cam)
        Xc = R @ P + t
        x, y = fx * Xc[0] / Xc[2] + cx, fy * Xc[1] / Xc[2] + cy
        px, py = int(math.floor(x)), int(math.floor(y))
        cam.cx = float(np.float32(cx + (px + 0.5 - x)))
        cam.cy = float(np.float32(cy + (py + 0.5 - y)))
        if not (0 <= px < 128 and 0 <= py < 128):
            continue
        w = orc.pixel_walk(s, cam, orc.Opts(chi2=9.0), px, py)
        assert len(w["id"]) == 1, trial
        # principal point rounded to float32: position error <= 1e-5 px
        assert abs(w["u"][0] - u0) < 2e-4 and abs(w["v"][0] - v0) < 2e-4, (trial, w["u"], u0, w["v"], v0)


def pin_two_surfels():
    """Eq. (1) for two overlapping surfels: C = c1 a1 + c2 a2 (1 - a1), T = (1-a1)(1-a2)."""
    s1, x1 = fronto_surfel(CAM, 0.05, 0.02, 2.0, 0.3, 0.3, 0.6, rgb=(1.0, 0.0, 0.0))
    s2, x2 = fronto_surfel(CAM, -0.03, 0.01, 2.5, 0.4, 0.25, 0.7, rgb=(0.0, 1.0, 0.0))
    s = concat(s2, s1)  # id 0 is the far one: order must come from depth, not id
    out = orc.render(s, CAM, orc.Opts())
    pix = out["pixels"].astype(float)
    a1, d1 = closed_form_alpha(CAM, x1, 0.3, 0.3, 0.6, pix[:, 0], pix[:, 1])
    a2, d2 = closed_form_alpha(CAM, x2, 0.4, 0.25, 0.7, pix[:, 0], pix[:, 1])
    both = (d1 < 8.9) & (d2 < 8.9) & (a1 > 1.01 / 255) & (a2 > 1.01 / 255)
    assert both.sum() > 100
    a1, a2 = np.minimum(a1, 0.99), np.minimum(a2, 0.99)
    assert np.max(np.abs(out["rgb"][both, 0] - a1[both])) < 1e-12
    assert np.max(np.abs(out["rgb"][both, 1] - a2[both] * (1 - a1[both]))) < 1e-12
    assert np.max(np.abs(out["T"][both] - (1 - a1[both]) * (1 - a2[both]))) < 1e-12


def pin_termination():
    """Five stacked opaque surfels: compositing stops after the surfel that
    takes T below 1e-4 (hand-computed count)."""
    layers = [fronto_surfel(CAM, 0.0, 0.0, 2.0 + 0.1 * i, 0.5, 0.5, 0.95) for i in range(5)]
    s = concat(*[l[0] for l in layers])
    px, py = 64, 64
    alphas = []
    for (_, xc) in layers:
        a, _ = closed_form_alpha(CAM, xc, 0.5, 0.5, 0.95, float(px), float(py))
        alphas.append(min(float(a), 0.99))
    T, n = 1.0, 0
    for a in alphas:
        T *= 1 - a
        n += 1
        if T < 1e-4:
            break
    out = orc.render(s, CAM, orc.Opts(), pixels=np.array([[px, py]]))
    assert out["ncontrib"][0] == n, (out["ncontrib"][0], n)
    assert abs(out["T"][0] - T) < 1e-15


def pin_partition_of_unity(w=None):
    """sum_j omega_j + T_final = 1 at every pixel."""
    w = w or sg.dense_box(n=3000)
    out = orc.render(w.surfels, w.cameras[0], orc.Opts(top_k=8), feat=w.features)
    assert np.max(np.abs(out["sumw"] + out["T"] - 1.0)) < 1e-12
    assert out["ncontrib"].max() > 8


def pin_topk_special_cases(w=None):
    """K >= #contributors gives the dense result bit for bit; K=1 keeps the
    largest weight; general K keeps the K largest weights (library sort)."""
    w = w or sg.dense_box(n=3000)
    cam = w.cameras[0]
    dense = orc.render(w.surfels, cam, orc.Opts(top_k=0), feat=w.features)
    big = orc.render(w.surfels, cam, orc.Opts(top_k=100000), feat=w.features)
    assert np.array_equal(dense["F"], big["F"])
    b = orc.bin_view(w.surfels, cam, orc.Opts())
    rich = np.nonzero(dense["ncontrib"] > 8)[0][:40]
    assert len(rich) >= 10
    feats = w.features.astype(np.float64)
    for K in (1, 3, 8):
        opts = orc.Opts(top_k=K)
        out = orc.render(w.surfels, cam, opts, feat=w.features, pixels=dense["pixels"][rich], b=b)
        for j, p in enumerate(rich):
            px, py = dense["pixels"][p]
            c = orc.pixel_walk(w.surfels, cam, opts, px, py, b=b)
            om = c["alpha"] * c["T"]
            order = np.argsort(-om, kind="stable")  # ties: earlier position first
            expect = set(c["id"][order[:K]].tolist())
            got = set(out["topk"][j][out["topk"][j] >= 0].tolist())
            assert got == expect, (K, p, got, expect)
            if K == 1:
                i = int(c["id"][order[0]])
                assert np.max(np.abs(out["F"][j] - om[order[0]] * feats[i])) < 1e-12


def pin_coverage(w=None, modes=(orc.SPHERE, orc.AABB, orc.EXACT), opacity_radius=False, lowpass=False):
    """Brute force: every (pixel, surfel) that contributes in FP64 has the
    surfel listed in that pixel's tile (all modes); EXACT <= AABB <= SPHERE."""
    w = w or sg.dense_box(n=3000)
    cam = w.cameras[0]
    n = w.surfels.n
    tiles_x = (cam.width + 15) // 16
    sets = {}
    for mode in modes:
        opts = orc.Opts(mode=mode, top_k=100000, opacity_radius=opacity_radius, lowpass=lowpass)
        keys, vals = orc.emit_pairs(w.surfels, [cam], opts)
        code = (keys >> np.uint64(32)).astype(np.int64) * n + vals.astype(np.int64)
        sets[mode] = np.unique(code)
        out = orc.render(w.surfels, cam, opts)
        pix = out["pixels"]
        K = out["topk"].shape[1]
        assert out["ncontrib"].max() <= K
        tile = (pix[:, 1] // 16) * tiles_x + (pix[:, 0] // 16)
        tk = out["topk"]
        m = tk >= 0
        need = (np.repeat(tile[:, None], K, 1)[m]).astype(np.int64) * n + tk[m].astype(np.int64)
        missing = ~np.isin(need, sets[mode])
        assert not missing.any(), (mode, int(missing.sum()))
    if len(modes) == 3:
        assert np.isin(sets[orc.EXACT], sets[orc.AABB]).all()
        assert np.isin(sets[orc.AABB], sets[orc.SPHERE]).all()
        assert len(sets[orc.EXACT]) < len(sets[orc.AABB]) < len(sets[orc.SPHERE])


def pin_conic_bounds(w=None, samples=96):
    """The exact AABB of the projected ellipse matches 10^4+ boundary points of
    the disc projected by hand (FP64)."""
    w = w or sg.dense_box(n=3000)
    cam = w.cameras[0]
    R, t, fx, fy, cx, cy = _cam_f64(cam)
    b = orc.bin_view(w.surfels, cam, orc.Opts(mode=orc.AABB))
    vis = np.nonzero(b["visible"])[0][:400]
    th = np.linspace(0, 2 * np.pi, samples, endpoint=False)
    s = w.surfels
    for i in vis:
        r = math.sqrt(float(b["r2"][i]) * (1.0 + 1.0 / 1024.0))
        mu, tu, tv = (getattr(s, f)[i].astype(np.float64) for f in ("mu", "tu", "tv"))
        su, sv = s.scale[i].astype(np.float64)
        P = mu[None] + (r * np.cos(th) * su)[:, None] * tu[None] + (r * np.sin(th) * sv)[:, None] * tv[None]
        Xc = P @ R.T + t
        x = fx * Xc[:, 0] / Xc[:, 2] + cx
        y = fy * Xc[:, 1] / Xc[:, 2] + cy
        ex, ey, A00, A01, A11, hx, hy = b["ell"][i][:7].astype(np.float64)
        tol = 1e-3 * max(1.0, hx, hy)
        assert x.min() >= ex - hx - tol and x.max() <= ex + hx + tol, (i, x.min(), x.max(), ex, hx)
        assert y.min() >= ey - hy - tol and y.max() <= ey + hy + tol, (i,)
        assert x.max() >= ex + hx - 5e-3 * hx - tol and x.min() <= ex - hx + 5e-3 * hx + tol
        assert y.max() >= ey + hy - 5e-3 * hy - tol and y.min() <= ey - hy + 5e-3 * hy + tol


def pin_ranges():
    """Per-tile ranges of the sorted keys equal a brute-force count per tile."""
    w = sg.dense_box(n=2000)
    cams = [w.cameras[0], sg.look_camera((0.5, -5.5, 1.2), 0.2, 96, 80, 90.0)]
    opts = orc.Opts(mode=orc.EXACT)
    keys, vals = orc.emit_pairs(w.surfels, cams, opts)
    sk, sv = orc.sort_pairs(keys, vals)
    nt = sum(orc.tiles_per_view(cams, opts))
    rg = orc.tile_ranges(sk, nt)
    counts = np.bincount((keys >> np.uint64(32)).astype(np.int64), minlength=nt)
    assert np.array_equal((rg[:, 1] - rg[:, 0]).astype(np.int64), counts)
    assert np.all(np.diff(sk.astype(np.float64)) >= 0) or np.all(sk[1:] >= sk[:-1])


def pin_rho():
    """rho(o) is an upper bound of 2 ln(255 o) within 2e-3 (library log)."""
    for o in np.concatenate([np.linspace(1 / 255, 1, 4001), np.float32(1 / 255) * (1 + np.arange(1, 50) * 1e-3)]):
        o32 = float(np.float32(o))
        if 255.0 * o32 <= 1.0:
            continue
        r = orc.rho_opacity(o32)
        ref = 2.0 * math.log(255.0 * o32)
        assert ref <= r <= ref + 2e-3, (o32, r, ref)


def fd_check(w, params_per_kind=12, seed=0, h_rel=1e-5, tol_rel=1e-6, tol_abs=2e-7, lowpass=False):
    """Central finite differences (Richardson-extrapolated from steps h and
    h/2, error O(h^4)) of the FP64 loss against the analytic gradient,
    skipping perturbations that change any discrete decision (with the
    low-pass filter, also which of its two terms wins)."""
    cam = w.cameras[0]
    s0 = w.surfels
    opts = orc.Opts(mode=orc.EXACT, top_k=w.top_k, lowpass=lowpass)
    npix = cam.width * cam.height
    D = w.features.shape[1]
    gC = sg.make_upstream(3 * npix, seed, 0).reshape(npix, 3).astype(np.float64)
    gF = sg.make_upstream(D * npix, seed, 1).reshape(npix, D).astype(np.float64)
    gT = sg.make_upstream(npix, seed, 2).astype(np.float64)
    b = orc.bin_view(s0, cam, opts)
    base = orc.render(s0, cam, opts, feat=w.features, b=b)
    g = orc.render_grad(s0, cam, opts, gC, feat=w.features, gF=gF, gT=gT, b=b)
    rng = np.random.default_rng(seed)
    used = np.unique(base["topk"][base["topk"] >= 0])
    assert len(used) > 20
    checked = 0
    worst = 0.0
    s64 = sg.Surfels(*(getattr(s0, f).astype(np.float64) for f in ("mu", "tu", "tv", "scale", "opacity", "rgb")))
    feat64 = w.features.astype(np.float64)
    kinds = [("mu", 3), ("tu", 3), ("tv", 3), ("scale", 2), ("opacity", 1), ("rgb", 3), ("feat", D)]
    for kind, width in kinds:
        for _ in range(params_per_kind):
            i = int(rng.choice(used))
            c = int(rng.integers(width))
            if kind == "feat":
                arr = feat64
            else:
                arr = getattr(s64, kind)
            flat = arr.reshape(arr.shape[0], -1)
            x0 = flat[i, c]
            h = h_rel * max(1.0, abs(x0))
            vals = []
            hashes_ok = True
            for step in (h, -h, 0.5 * h, -0.5 * h):
                flat[i, c] = x0 + step
                out = orc.render(s64, cam, opts, feat=feat64, b=b)
                hashes_ok &= bool(np.array_equal(out["hash"], base["hash"]))
                vals.append(orc.loss(out, gC, gF, gT))
            flat[i, c] = x0
            if not hashes_ok:
                continue
            d1 = (vals[0] - vals[1]) / (2 * h)
            d2 = (vals[2] - vals[3]) / h
            fd = (4.0 * d2 - d1) / 3.0
            an = float(g["feat" if kind == "feat" else kind].reshape(arr.shape[0], -1)[i, c])
            err = abs(fd - an)
            assert err <= tol_rel * abs(an) + tol_abs, (kind, i, c, fd, an)
            worst = max(worst, err / max(abs(an), 1e-12))
            checked += 1
    assert checked >= 4 * params_per_kind, checked
    return checked, worst


def _disc_boundary(s, i, r, cam, samples):
    """Points of surfel i's disc of radius r (in (u, v) units) at `samples`
    angles, in camera space (FP64, by hand)."""
    R, t, *_ = _cam_f64(cam)
    th = np.linspace(0, 2 * np.pi, samples, endpoint=False)
    mu, tu, tv = (getattr(s, f)[i].astype(np.float64) for f in ("mu", "tu", "tv"))
    su, sv = s.scale[i].astype(np.float64)
    P = mu[None] + (r * np.cos(th) * su)[:, None] * tu[None] + (r * np.sin(th) * sv)[:, None] * tv[None]
    return P @ R.T + t


def pin_near_plane(s=None, margin=1e-4, samples=8192):
    """Near-plane cull (reading: a surfel is culled unless its whole binning
    disc lies beyond z_near): brute force over the sampled boundary of the
    disc of radius r_b = sqrt(r^2 (1 + 2^-10)) -- a disc's nearest point is on
    its boundary -- decides visibility; straddles within `margin` of z_near
    are excused. The scene must contain surfels whose centre is beyond the
    plane while their disc crosses it, and surfels wholly beyond it."""
    s = s if s is not None else sg.near_plane().surfels
    opts = orc.Opts(mode=orc.AABB)
    b = orc.bin_view(s, CAM, opts)
    rb = math.sqrt(opts.chi2 * (1.0 + 1.0 / 1024.0))
    crossing = beyond = 0
    for i in range(s.n):
        Xc = _disc_boundary(s, i, rb, CAM, samples)
        zmin = Xc[:, 2].min()
        if abs(zmin - opts.z_near) < margin:
            continue
        if zmin < opts.z_near:
            assert not b["visible"][i], (i, zmin)
            centre_z = (_cam_f64(CAM)[0] @ s.mu[i].astype(np.float64) + _cam_f64(CAM)[1])[2]
            crossing += int(centre_z > opts.z_near)
        else:
            # wholly beyond the plane, centred in the image: must be kept
            assert b["visible"][i], (i, zmin)
            beyond += 1
    assert crossing >= 20 and beyond >= 20, (crossing, beyond)
    return crossing, beyond


def pin_sphere_radius(s=None, samples=4096, n_max=300):
    """SPHERE mode (the paper's isotropic bounding sphere): the square's
    half-width is the radius of the smallest circle about the ellipse centre
    that holds the projected binning disc, i.e. its semi-major axis. Checked
    against hand-projected boundary points: the centre is the midpoint of their
    x and y extremes, the radius their largest distance from it."""
    s = s if s is not None else concat(sg.near_plane(seed=12, n=200).surfels, sg.dense_box(n=3000).surfels)
    cam = CAM
    R, t, fx, fy, cx, cy = _cam_f64(cam)
    opts = orc.Opts(mode=orc.SPHERE)
    b = orc.bin_view(s, cam, opts)
    rb = math.sqrt(opts.chi2 * (1.0 + 1.0 / 1024.0))
    vis = np.nonzero(b["visible"])[0][:n_max]
    rotated = 0
    for i in vis:
        Xc = _disc_boundary(s, i, rb, cam, samples)
        x = fx * Xc[:, 0] / Xc[:, 2] + cx
        y = fy * Xc[:, 1] / Xc[:, 2] + cy
        ex, ey = 0.5 * (x.min() + x.max()), 0.5 * (y.min() + y.max())
        semi = np.sqrt((x - ex) ** 2 + (y - ey) ** 2).max()
        hx, hy, extx, exty = (float(v) for v in b["ell"][i][5:9])
        assert extx == exty, i
        tol = 2e-3 * max(1.0, semi)
        assert abs(extx - semi) <= tol, (i, extx, semi, hx, hy)
        rotated += int(semi > max(hx, hy) * 1.01 + tol)
    assert len(vis) >= 100 and rotated >= 20, (len(vis), rotated)
    return len(vis), rotated
