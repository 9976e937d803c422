"""Python face of the CPU oracle (test infrastructure only).

Wraps oracle/psi_oracle.c through ctypes and adds the few steps that are
library routines: the stable sort of the key array (numpy's stable argsort),
the per-tile ranges, and the FP64 query contraction of the decode step.

Every function takes plain numpy arrays produced by the seeded scene
generator; nothing here imports the CUDA package.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

SPHERE, AABB, EXACT = 0, 1, 2
ALPHA_MIN = 1.0 / 255.0
T_EPS = 1e-4

_lib = None
_plant = 0


def use_variant(plant: int = 0) -> None:
    """Switch to a deliberately wrong build (plant > 0) or back to the real one.
    Only the test that checks the pins catch planted mistakes calls this."""
    global _lib, _plant
    _plant = int(plant)
    _lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build(plant=_plant)
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, f32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
        L.or_bin_view.argtypes = [i64, P, P, P, P, P, P, f32, f32, i32, i32, i32, i32, i32, P, P, P, P, P]
        L.or_bin_view.restype = None
        L.or_emit_view.argtypes = [i64, P, P, P, P, P, P, f32, f32, i32, i32, i32, i32, i32,
                                   ctypes.c_uint32, ctypes.c_uint32, P, P, i64]
        L.or_emit_view.restype = i64
        L.or_rho_opacity.argtypes = [f32]
        L.or_rho_opacity.restype = f32
        L.or_render.argtypes = [i64, P, P, P, P, P, P, P, i32, P, i32, P, P, i64, P, i32, f64, i32,
                                P, P, P, P, P, P, P, P]
        L.or_render.restype = None
        L.or_render_grad.argtypes = [i64, P, P, P, P, P, P, P, i32, P, i32, P, P, i64, P, i32, f64, i32,
                                     P, P, P, P, P, P, P, P, P, P]
        L.or_render_grad.restype = None
        L.or_pixel_walk.argtypes = [i64, P, P, P, P, P, P, i32, P, P, i32, i32, i32, f64, i32, P, P, P, i32]
        L.or_pixel_walk.restype = i32
        L.or_num_threads.restype = i32
        L.or_set_threads.argtypes = [i32]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class Opts:
    """Render options shared by the oracle and the CUDA path (same meaning)."""
    mode: int = EXACT
    top_k: int = 0          # 0 = dense features
    chi2: float = 9.0
    z_near: float = 0.2
    opacity_radius: bool = False
    tile_w: int = 16
    tile_h: int = 16
    t_eps: float = T_EPS
    lowpass: bool = False   # 2DGS object-space low-pass filter: rho = min(u^2+v^2, 2|x-c|^2)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def rho_opacity(o: float) -> float:
    return float(lib().or_rho_opacity(float(o)))


def _surf32(s):
    return (_c(s.mu, np.float32), _c(s.tu, np.float32), _c(s.tv, np.float32), _c(s.scale, np.float32),
            _c(s.opacity, np.float32))


def bin_view(s, cam, opts: Opts):
    """Discrete (pinned float32) per-surfel results for one camera."""
    mu, tu, tv, sc, o = _surf32(s)
    n = s.n
    camv = _c(cam.as_array(), np.float32)
    count = np.zeros(n, np.uint32)
    dbits = np.zeros(n, np.uint32)
    r2 = np.zeros(n, np.float32)
    rect = np.zeros((n, 4), np.int32)
    ell = np.zeros((n, 9), np.float32)
    lib().or_bin_view(n, _p(mu), _p(tu), _p(tv), _p(sc), _p(o), _p(camv), opts.chi2, opts.z_near,
                      int(opts.opacity_radius), int(opts.mode), int(opts.lowpass), opts.tile_w, opts.tile_h,
                      _p(count), _p(dbits), _p(r2), _p(rect), _p(ell))
    return dict(count=count, depth_bits=dbits, r2=r2, rect=rect, ell=ell, visible=rect[:, 0] >= 0)


def tiles_per_view(cams, opts: Opts):
    return [((c.width + opts.tile_w - 1) // opts.tile_w) * ((c.height + opts.tile_h - 1) // opts.tile_h) for c in cams]


def emit_pairs(s, cams, opts: Opts):
    """Unsorted (key, value) pairs of all views in emission order.

    value = view * N + surfel; key = global tile << 32 | float bits of depth."""
    mu, tu, tv, sc, o = _surf32(s)
    n = s.n
    keys_all, vals_all = [], []
    base = 0
    tpv = tiles_per_view(cams, opts)
    for v, cam in enumerate(cams):
        camv = _c(cam.as_array(), np.float32)
        b = bin_view(s, cam, opts)
        cap = int(b["count"].sum())
        keys = np.zeros(max(cap, 1), np.uint64)
        vals = np.zeros(max(cap, 1), np.uint32)
        got = lib().or_emit_view(n, _p(mu), _p(tu), _p(tv), _p(sc), _p(o), _p(camv), opts.chi2, opts.z_near,
                                 int(opts.opacity_radius), int(opts.mode), int(opts.lowpass), opts.tile_w,
                                 opts.tile_h, base, v * n, _p(keys), _p(vals), cap)
        assert got == cap, (got, cap)
        keys_all.append(keys[:cap])
        vals_all.append(vals[:cap])
        base += tpv[v]
    return np.concatenate(keys_all), np.concatenate(vals_all)


def sort_pairs(keys, vals):
    """Stable sort by key (library routine: numpy's stable radix/merge sort)."""
    perm = np.argsort(keys, kind="stable")
    return keys[perm], vals[perm]


def tile_ranges(sorted_keys, n_tiles_total):
    """[n_tiles, 2] (start, end) of each global tile in the sorted key array."""
    tiles = (sorted_keys >> np.uint64(32)).astype(np.int64)
    idx = np.arange(n_tiles_total, dtype=np.int64)
    start = np.searchsorted(tiles, idx, side="left")
    end = np.searchsorted(tiles, idx, side="right")
    return np.stack([start, end], 1).astype(np.uint32)


def canonical_order(b):
    """Non-culled surfels of one view sorted by (float32 depth bits, id)."""
    ids = np.nonzero(b["visible"])[0]
    return ids[np.lexsort((ids, b["depth_bits"][ids]))].astype(np.int32)


def _surf64(s):
    return tuple(_c(a, np.float64) for a in (s.mu, s.tu, s.tv, s.scale, s.opacity, s.rgb))


def all_pixels(cam):
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    return np.stack([xs.reshape(-1), ys.reshape(-1)], 1).astype(np.int32)


def render(s, cam, opts: Opts, feat=None, pixels=None, b=None):
    """FP64 brute-force render of the given pixels ([P,2] x,y; default all).

    feat: [N,D] array of the (dequantised) feature values, or None.
    Returns dict with rgb [P,3], T [P], F [P,D], topk [P,K] (surfel ids in list
    order, -1 padded), ncontrib, sumw, diag [P,6], hash."""
    if b is None:
        b = bin_view(s, cam, opts)
    order = canonical_order(b)
    r2 = b["r2"].astype(np.float64)
    pix = all_pixels(cam) if pixels is None else _c(pixels, np.int32)
    npix = pix.shape[0]
    mu, tu, tv, sc, o, rgb = _surf64(s)
    D = 0 if feat is None else int(feat.shape[1])
    f64 = None if feat is None else _c(feat, np.float64)
    K = int(opts.top_k)
    out = dict(rgb=np.zeros((npix, 3)), T=np.zeros(npix), F=np.zeros((npix, max(D, 1))),
               topk=np.full((npix, max(K, 1)), -1, np.int32), ncontrib=np.zeros(npix, np.int32),
               sumw=np.zeros(npix), diag=np.zeros((npix, 6)), hash=np.zeros(npix, np.uint64))
    camv = _c(cam.as_array(), np.float64)
    lib().or_render(s.n, _p(mu), _p(tu), _p(tv), _p(sc), _p(o), _p(rgb), _p(f64), D, _p(order), len(order),
                    _p(r2), _p(camv), npix, _p(pix), K, opts.t_eps, int(opts.lowpass),
                    _p(out["rgb"]), _p(out["T"]), _p(out["F"]) if D else None,
                    _p(out["topk"]) if K > 0 else None, _p(out["ncontrib"]), _p(out["sumw"]), _p(out["diag"]),
                    _p(out["hash"]))
    if not D:
        out["F"] = np.zeros((npix, 0))
    out["pixels"] = pix
    return out


def pixel_walk(s, cam, opts: Opts, px: int, py: int, b=None, cap: int = 4096):
    """Contributors of one pixel, front to back: dict(id, u, v, alpha, T, sel)."""
    if b is None:
        b = bin_view(s, cam, opts)
    order = canonical_order(b)
    r2 = b["r2"].astype(np.float64)
    mu, tu, tv, sc, o, rgb = _surf64(s)
    camv = _c(cam.as_array(), np.float64)
    ids = np.zeros(cap, np.int32)
    uvat = np.zeros((cap, 4))
    sel = np.zeros(cap, np.uint8)
    cnt = lib().or_pixel_walk(s.n, _p(mu), _p(tu), _p(tv), _p(sc), _p(o), _p(order), len(order), _p(r2), _p(camv),
                              int(px), int(py), int(opts.top_k), opts.t_eps, int(opts.lowpass), _p(ids), _p(uvat), _p(sel), cap)
    cnt = min(cnt, cap)
    return dict(id=ids[:cnt], u=uvat[:cnt, 0], v=uvat[:cnt, 1], alpha=uvat[:cnt, 2], T=uvat[:cnt, 3],
                sel=sel[:cnt].astype(bool))


def render_grad(s, cam, opts: Opts, gC, feat=None, gF=None, gT=None, pixels=None, b=None):
    """FP64 gradient of L = sum gC.C + gF.F + gT.T over the given pixels."""
    if b is None:
        b = bin_view(s, cam, opts)
    order = canonical_order(b)
    r2 = b["r2"].astype(np.float64)
    pix = all_pixels(cam) if pixels is None else _c(pixels, np.int32)
    npix = pix.shape[0]
    mu, tu, tv, sc, o, rgb = _surf64(s)
    D = 0 if feat is None else int(feat.shape[1])
    f64 = None if feat is None else _c(feat, np.float64)
    n = s.n
    g = dict(mu=np.zeros((n, 3)), tu=np.zeros((n, 3)), tv=np.zeros((n, 3)), scale=np.zeros((n, 2)),
             opacity=np.zeros(n), rgb=np.zeros((n, 3)), feat=np.zeros((n, max(D, 1))))
    camv = _c(cam.as_array(), np.float64)
    gC = _c(gC, np.float64).reshape(npix, 3)
    gF = None if (gF is None or D == 0) else _c(gF, np.float64).reshape(npix, D)
    gT = None if gT is None else _c(gT, np.float64).reshape(npix)
    lib().or_render_grad(n, _p(mu), _p(tu), _p(tv), _p(sc), _p(o), _p(rgb), _p(f64), D, _p(order), len(order),
                         _p(r2), _p(camv), npix, _p(pix), int(opts.top_k), opts.t_eps, int(opts.lowpass),
                         _p(gC), _p(gF), _p(gT), _p(g["mu"]), _p(g["tu"]), _p(g["tv"]), _p(g["scale"]),
                         _p(g["opacity"]), _p(g["rgb"]), _p(g["feat"]) if D else None)
    if not D:
        g["feat"] = np.zeros((n, 0))
    return g


def loss(out, gC, gF=None, gT=None):
    """L = sum gC.C + gF.F + gT.T of a render result (FP64)."""
    L = float(np.sum(out["rgb"] * np.asarray(gC, np.float64).reshape(out["rgb"].shape)))
    if gF is not None and out["F"].shape[1]:
        L += float(np.sum(out["F"] * np.asarray(gF, np.float64).reshape(out["F"].shape)))
    if gT is not None:
        L += float(np.sum(out["T"] * np.asarray(gT, np.float64).reshape(out["T"].shape)))
    return L


def decode(F, Q, T, empty_eps: float = 1e-4):
    """FP64 query contraction (library matmul) and argmax, lowest index on ties.

    F: [P,D] feature values (as the GPU stored them), Q: [Q,D], T: [P].
    Returns (ids [P] int32, logits [P,Q] float64, gap [P] top-2 logit gap)."""
    L = np.asarray(F, np.float64) @ np.asarray(Q, np.float64).T
    ids = np.argmax(L, axis=1).astype(np.int32)
    if L.shape[1] > 1:
        part = -np.sort(-L, axis=1)
        gap = part[:, 0] - part[:, 1]
    else:
        gap = np.full(L.shape[0], np.inf)
    empty = (1.0 - np.asarray(T, np.float64)) < empty_eps
    ids[empty] = -1
    return ids, L, gap


def surfel_labels(feat, queries, q_mu, q_cov, centres, plant: int = 0):
    """Per-surfel instance label distribution (Sec. 4.1, Eqs. 4-7), FP64.

    feat [N, D] (the stored feature values), queries [Q, D] (query features
    f_q), q_mu [Q, 3] and q_cov [Q, 3, 3] (each query's spatial Gaussian),
    centres [N, 3] (surfel centres p_g). For every query q and surfel g:
      S(f_q, f_g) = sigmoid(f_q^T f_g)                        (Eq. 4)
      D(p_q, p_g) = phi_q(p_g) / phi_q(p_q), with phi_q the density of
                    N(mu_q, Sigma_q) and p_q = mu_q its centre   (Eq. 5)
      A(q, g)     = S D                                       (Eq. 6)
      l_ins(g)    = softmax over the Q queries of A(., g)     (Eq. 7)
    The ratio of densities leaves exp(-(p_g - mu_q)^T Sigma_q^-1 (p_g - mu_q) / 2).
    Returns [N, Q] float64. `plant` > 0 builds a deliberately wrong variant
    (only the test that checks the pins uses it)."""
    f = np.asarray(feat, np.float64)
    qf = np.asarray(queries, np.float64)
    mu = np.asarray(q_mu, np.float64)
    cov = np.asarray(q_cov, np.float64)
    p = np.asarray(centres, np.float64)
    z = f @ qf.T
    S = z if plant == 4 else 1.0 / (1.0 + np.exp(-z))
    prec = cov if plant == 3 else np.linalg.inv(cov)
    d = p[:, None, :] - mu[None, :, :]
    m2 = np.einsum("nqi,qij,nqj->nq", d, prec, d)
    D = np.exp(-m2) if plant == 1 else np.exp(-0.5 * m2)
    A = S * D
    axis = 0 if plant == 2 else 1
    e = np.exp(A - A.max(axis=axis, keepdims=True))
    return e / e.sum(axis=axis, keepdims=True)


def label_ids(I, T, empty_eps: float = 1e-4):
    """Pixel instance identity from the rendered label mixture I [P, Q]
    (Eq. 8): argmax over queries, lowest index on ties, -1 where nothing was
    rendered. Returns (ids [P] int32, gap [P] top-2 margin)."""
    I = np.asarray(I, np.float64)
    ids = np.argmax(I, axis=1).astype(np.int32)
    part = -np.sort(-I, axis=1)
    gap = part[:, 0] - part[:, 1] if I.shape[1] > 1 else np.full(I.shape[0], np.inf)
    ids[(1.0 - np.asarray(T, np.float64)) < empty_eps] = -1
    return ids, gap


def surfel_regularisers(s, node_of, node_mu, node_n, lambda_n: float, plant: int = 0):
    """Geometric and anisotropy regularisers of the joint objective (Sec. 4.2), FP64.

    For surfel i with an assigned planar prior k = node_of[i] (>= 0; -1: none),
    prior centre m_k and unit normal nhat_k:
      d_i   = |(mu_i - m_k) . nhat_k|                  point-to-plane distance
      L_geo = sum_i d_i + lambda_n (1 - |n_i . nhat_k|),  n_i = t_u x t_v / |t_u x t_v|
      L_iso = sum_i (s_i1 - s_i2)^2
    Returns (L_geo, L_iso, grads) with grads the gradients of L_geo (keys
    mu, tu, tv) and of L_iso (key scale), each [N, ...] float64, written by
    hand from the chain rule. `plant` > 0 builds a deliberately wrong variant
    (only the pin test uses it)."""
    mu = np.asarray(s.mu, np.float64)
    tu = np.asarray(s.tu, np.float64)
    tv = np.asarray(s.tv, np.float64)
    sc = np.asarray(s.scale, np.float64)
    k = np.asarray(node_of, np.int64)
    has = k >= 0
    m = np.asarray(node_mu, np.float64)[np.where(has, k, 0)]
    nh = np.asarray(node_n, np.float64)[np.where(has, k, 0)]
    c = np.cross(tu, tv)
    cn = np.linalg.norm(c, axis=1, keepdims=True)
    n = c / cn
    off = np.sum((mu - m) * nh, axis=1)
    dot = np.sum(n * nh, axis=1)
    term_n = (1.0 - dot) if plant == 2 else (1.0 - np.abs(dot))
    L_geo = float(np.sum(np.where(has, np.abs(off) + lambda_n * term_n, 0.0)))
    diff = sc[:, 0] - sc[:, 1]
    L_iso = float(np.sum(diff * diff)) if plant != 3 else float(np.sum(np.abs(diff)))
    g = {}
    g["mu"] = np.where(has[:, None], np.sign(off)[:, None] * nh, 0.0)
    gn = np.where(has[:, None], -lambda_n * (np.ones_like(dot) if plant == 2 else np.sign(dot))[:, None] * nh, 0.0)
    # n = c/|c|: dL/dc = (I - n n^T) dL/dn / |c|; c = tu x tv: dL/dtu = tv x dL/dc, dL/dtv = dL/dc x tu
    gc = (gn - np.sum(gn * n, axis=1, keepdims=True) * n) / cn
    if plant == 1:
        gc = gn / cn
    g["tu"] = np.cross(tv, gc)
    g["tv"] = np.cross(gc, tu)
    g["scale"] = np.stack([2.0 * diff, -2.0 * diff], axis=1)
    return L_geo, L_iso, g


def quat_frames(q, plant: int = 0):
    """Tangent frame of a quaternion-parameterised surfel (the 2DGS form), FP64.

    q [N, 4] = (w, x, y, z), not necessarily unit: R = R(q / |q|) and
    t_u, t_v are its first two columns (the third is the surfel normal).
    Returns (tu [N,3], tv [N,3])."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    if plant == 1:
        x = -x
    tu = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], axis=1)
    tv = np.stack([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)], axis=1)
    return tu, tv


def quat_frames_grad(q, g_tu, g_tv):
    """dL/dq from dL/dt_u, dL/dt_v through quat_frames (normalisation
    included), written from the partial derivatives of R's columns."""
    q = np.asarray(q, np.float64)
    nq = np.linalg.norm(q, axis=1, keepdims=True)
    u = q / nq
    w, x, y, z = u[:, 0], u[:, 1], u[:, 2], u[:, 3]
    gu = np.asarray(g_tu, np.float64)
    gv = np.asarray(g_tv, np.float64)
    zero = np.zeros_like(w)
    # d t_u / d(w, x, y, z) and d t_v / d(w, x, y, z), each [N, 3]
    du = [np.stack(c, 1) for c in ((zero, 2 * z, -2 * y), (zero, 2 * y, 2 * z), (-4 * y, 2 * x, -2 * w),
                                   (-4 * z, 2 * w, 2 * x))]
    dv = [np.stack(c, 1) for c in ((-2 * z, zero, 2 * x), (2 * y, -4 * x, 2 * w), (2 * x, zero, 2 * z),
                                   (-2 * w, -4 * z, 2 * y))]
    gq_hat = np.stack([np.sum(gu * du[k], 1) + np.sum(gv * dv[k], 1) for k in range(4)], axis=1)
    # through q / |q|
    return (gq_hat - np.sum(gq_hat * u, axis=1, keepdims=True) * u) / nq


def surfel_geometry(s, cam, plant: int = 0):
    """Per-surfel geometry table for depth and normal maps, FP64.

    For surfel i seen by `cam`: z_i = (R mu_i + t)_z, the camera depth of its
    centre, and n_i = R (t_u x t_v) / |t_u x t_v|, its unit normal in camera
    coordinates, turned to face the camera (negated where n . x_c > 0; an
    edge-on surfel keeps its sign). Returns [N, 4] = (z, n_x, n_y, n_z).
    Blended with the compositing weights like any dense feature, the columns
    give the expected depth sum_j omega_j z_j and normal sum_j omega_j n_j
    maps of the 2D-surfel model (Sec. 3.1). `plant` > 0 builds a deliberately
    wrong variant (only the pin test uses it)."""
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    tt = np.asarray(cam.t, np.float64).reshape(3)
    xc = np.asarray(s.mu, np.float64) @ R.T + tt
    c = np.cross(np.asarray(s.tu, np.float64), np.asarray(s.tv, np.float64))
    n = (c / np.linalg.norm(c, axis=1, keepdims=True)) @ R.T
    if plant != 1:
        n = np.where((np.sum(n * xc, axis=1) > 0.0)[:, None], -n, n)
    return np.concatenate([xc[:, 2:3], n], axis=1)


def surfel_geometry_grad(s, cam, g, plant: int = 0):
    """dL/dmu, dL/dt_u, dL/dt_v of L = sum g . surfel_geometry (g [N, 4]),
    written from the chain rule (the sign choice is piecewise constant)."""
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    tt = np.asarray(cam.t, np.float64).reshape(3)
    tu = np.asarray(s.tu, np.float64)
    tv = np.asarray(s.tv, np.float64)
    g = np.asarray(g, np.float64)
    xc = np.asarray(s.mu, np.float64) @ R.T + tt
    c = np.cross(tu, tv)
    cn = np.linalg.norm(c, axis=1, keepdims=True)
    nw = c / cn
    flip = np.sum((nw @ R.T) * xc, axis=1) > 0.0
    g_mu = g[:, 0:1] * R[2][None, :]                      # z = R[2] . mu + t_z
    g_nc = np.where(flip[:, None], -g[:, 1:4], g[:, 1:4])
    g_nw = g_nc @ R                                       # n_c = R n_w
    g_c = g_nw / cn if plant == 2 else (g_nw - np.sum(g_nw * nw, axis=1, keepdims=True) * nw) / cn
    return {"mu": g_mu, "tu": np.cross(tv, g_c), "tv": np.cross(g_c, tu)}


CHI2_99_2D = -2.0 * np.log(0.01)  # chi-square quantile of 2 DOF at 99 %: the 99 % disc has radius 3.035 sigma


def attn_pos_enc(mu, C: int):
    """Positional encoding psi(mu) [N, C] of surfel centres (Sec. 4.1): channel
    c encodes axis c mod 3 with sin (t = c // 3 even) or cos (t odd) at the
    frequency w_k = 10000^(-6k/C), k = t // 2 (a sinusoidal encoding per
    axis; the paper names psi without fixing it)."""
    mu = np.asarray(mu, np.float64)
    c = np.arange(C)
    a = c % 3
    t = c // 3
    w = np.exp(-np.log(10000.0) * 6.0 * (t // 2) / C)
    arg = mu[:, a] * w[None, :]
    return np.where((t % 2 == 0)[None, :], np.sin(arg), np.cos(arg))


def frustum_active(s, cam, z_near: float):
    """Surfels whose 99 % confidence disc (radius sqrt(chi2_2(0.99)) max(s_u,
    s_v) around mu, bounded by its sphere) meets the view frustum: the
    sphere is not wholly behind the near plane or outside a side plane of
    the image rectangle. Returns (active [N] bool, margin [N]: the smallest
    signed plane distance plus the radius, in metres)."""
    mu = np.asarray(s.mu, np.float64)
    sc = np.asarray(s.scale, np.float64)
    R, t = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)
    x = mu @ R.T + t
    r = np.sqrt(CHI2_99_2D) * sc.max(axis=1)
    fx, fy, cx, cy, W, H = cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height
    planes = [np.array([0.0, 0.0, 1.0, -z_near]),           # z >= z_near
              np.array([fx, 0.0, cx, 0.0]),                  # x / z >= -cx / fx
              np.array([-fx, 0.0, W - cx, 0.0]),             # x / z <= (W - cx) / fx
              np.array([0.0, fy, cy, 0.0]),                  # y / z >= -cy / fy
              np.array([0.0, -fy, H - cy, 0.0])]             # y / z <= (H - cy) / fy
    d = np.stack([(x @ p[:3] + p[3]) / np.linalg.norm(p[:3]) for p in planes], axis=1)
    margin = (d + r[:, None]).min(axis=1)
    return margin >= 0.0, margin


def frustum_attention(s, feat, cam, z_near, Q, WQ, WK, WV, plant: int = 0):
    """Frustum-constrained cross-attention (Sec. 4.1), FP64: over the active
    surfels j, K_j = f_j + psi(mu_j), V_j = f_j,
      e_ij = (Q_i W_Q)(K_j W_K)^T / sqrt(d),  Q'_i = softmax_j(e_ij) (V_j W_V).
    feat [N, C] (stored values), Q [n_q, C], W_Q/W_K/W_V [C, d].
    Returns (Q' [n_q, d], active [N], margin [N])."""
    f = np.asarray(feat, np.float64)
    active, margin = frustum_active(s, cam, z_near)
    C = f.shape[1]
    if not active.any():  # reading: an empty active set attends to nothing, Q' = 0
        return np.zeros((np.asarray(Q).shape[0], np.asarray(WV).shape[1])), active, margin
    K = f + attn_pos_enc(s.mu, C)
    q = np.asarray(Q, np.float64) @ np.asarray(WQ, np.float64)
    k = K[active] @ np.asarray(WK, np.float64)
    v = f[active] @ np.asarray(WV, np.float64)
    d = q.shape[1]
    e = q @ k.T if plant == 1 else q @ k.T / np.sqrt(d)
    axis = 0 if plant == 2 else 1
    e = e - e.max(axis=axis, keepdims=True)
    P = np.exp(e)
    P /= P.sum(axis=axis, keepdims=True)
    return P @ v, active, margin


def frustum_attention_grad(s, feat, cam, z_near, Q, WQ, WK, WV, G):
    """Gradients of L = <G, Q'> through frustum_attention (Sec. 4.1), FP64,
    written by hand from the chain rule:
      dP = G v^T, dv = P^T G, de = P (dP - rowsum(P dP)), dq = de k / sqrt(d),
      dk = de^T q / sqrt(d), dQ = dq W_Q^T, dW_Q = Q^T dq, dK = dk W_K^T,
      dW_K = K^T dk, dV = dv W_V^T, dW_V = V^T dv,
      df = dK + dV, dmu_a = sum_c dK_c dpsi_c/dmu_a (active surfels only).
    Returns a dict with Q, WQ, WK, WV, feat [N, C], mu [N, 3]."""
    f = np.asarray(feat, np.float64)
    Q = np.asarray(Q, np.float64)
    WQ, WK, WV = (np.asarray(x, np.float64) for x in (WQ, WK, WV))
    G = np.asarray(G, np.float64)
    active, _ = frustum_active(s, cam, z_near)
    C = f.shape[1]
    mu = np.asarray(s.mu, np.float64)
    if not active.any():  # Q' = 0 identically: every gradient vanishes
        return {"Q": np.zeros_like(Q), "WQ": np.zeros_like(WQ), "WK": np.zeros_like(WK), "WV": np.zeros_like(WV),
                "feat": np.zeros_like(f), "mu": np.zeros_like(mu)}
    K = f + attn_pos_enc(mu, C)
    Ka, Va = K[active], f[active]
    q, k, v = Q @ WQ, Ka @ WK, Va @ WV
    d = q.shape[1]
    e = q @ k.T / np.sqrt(d)
    P = np.exp(e - e.max(axis=1, keepdims=True))
    P /= P.sum(axis=1, keepdims=True)
    dP = G @ v.T
    dv = P.T @ G
    de = P * (dP - np.sum(P * dP, axis=1, keepdims=True))
    dq = de @ k / np.sqrt(d)
    dk = de.T @ q / np.sqrt(d)
    out = {"Q": dq @ WQ.T, "WQ": Q.T @ dq, "WK": Ka.T @ dk, "WV": Va.T @ dv}
    dK = np.zeros_like(f)
    dV = np.zeros_like(f)
    dK[active] = dk @ WK.T
    dV[active] = dv @ WV.T
    out["feat"] = dK + dV
    # d psi / d mu: channel c depends on axis c mod 3 only
    c = np.arange(C)
    a, t = c % 3, c // 3
    w = np.exp(-np.log(10000.0) * 6.0 * (t // 2) / C)
    arg = mu[:, a] * w[None, :]
    dpsi = np.where((t % 2 == 0)[None, :], np.cos(arg), -np.sin(arg)) * w[None, :]
    dmu = np.zeros_like(mu)
    for ax in range(3):
        dmu[:, ax] = np.sum((dK * dpsi)[:, a == ax], axis=1)
    out["mu"] = dmu
    return out
