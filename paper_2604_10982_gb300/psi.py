"""ctypes binding of libpsi (include/psi.h): the same entry points, argument
marshalling only. Every step of the rendering path runs in the library's CUDA
kernels; PyTorch supplies device memory and the stream.

Loading fails loudly if the library has not been built (there is no CPU
fallback): build it with ``python -c "import __graft_entry__ as g; g.build()"``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PSI_LIBRARY=debug selects the bounds-checked build (libpsi_debug.so)
LIB_PATH = os.path.join(HERE, "_build", "libpsi_debug.so" if os.environ.get("PSI_LIBRARY") == "debug" else "libpsi.so")

PSI_OK, PSI_ERR_INVALID_ARG, PSI_ERR_CUDA, PSI_ERR_CAPACITY, PSI_ERR_TIMEOUT, PSI_ERR_UNSUPPORTED, PSI_ERR_BOUNDS = range(7)
SPHERE, AABB, EXACT = 0, 1, 2
F32, BF16, FP8_E4M3 = 0, 1, 2
KERNEL_BWD_FEAT, KERNEL_BWD_WALK = 1, 2  # enum psi_kernel_id
MAX_VIEWS = 64
RECORD_BYTES = 80
BIN_RECORD_BYTES = 32
BIN_RECORD_BYTES_LOWPASS = 48
MAX_TOPK = 32

_P = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class PsiSurfels(ctypes.Structure):
    _fields_ = [("mu", _P), ("tu", _P), ("tv", _P), ("scale", _P), ("opacity", _P), ("rgb", _P), ("n", _i64)]


class PsiCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", _i32), ("height", _i32)]


class PsiFeatures(ctypes.Structure):
    _fields_ = [("data", _P), ("scale", _P), ("dtype", _i32), ("dim", _i32)]


class PsiRenderOpts(ctypes.Structure):
    _fields_ = [("mode", _i32), ("top_k", _i32), ("chi2", ctypes.c_float), ("z_near", ctypes.c_float),
                ("opacity_radius", _i32), ("tile_w", _i32), ("tile_h", _i32), ("t_eps", ctypes.c_float),
                ("lowpass", _i32)]


class PsiFwdOut(ctypes.Structure):
    _fields_ = [("rgb", _P), ("T", _P), ("n_last", _P), ("F", _P), ("F_dtype", _i32), ("topk_ids", _P),
                ("topk_w", _P), ("argmax", _P)]


class PsiGrads(ctypes.Structure):
    _fields_ = [("mu", _P), ("tu", _P), ("tv", _P), ("scale", _P), ("opacity", _P), ("rgb", _P), ("feat", _P)]


_lib = None


class PsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"psi error {code}: {msg}")
        self.code = code


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpsi is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        sz = ctypes.c_size_t
        L.psi_ctx_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
        L.psi_ctx_destroy.argtypes = [_P]
        L.psi_ctx_destroy.restype = None
        L.psi_last_error.argtypes = [_P]
        L.psi_last_error.restype = ctypes.c_char_p
        L.psi_status_fetch.argtypes = [_P, _P, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]
        L.psi_default_opts.argtypes = [ctypes.POINTER(PsiRenderOpts)]
        L.psi_default_opts.restype = None
        L.psi_view_layout.argtypes = [ctypes.POINTER(PsiCamera), ctypes.c_int, ctypes.POINTER(PsiRenderOpts), _P, _P]
        for f in ("psi_intersect_workspace_size", "psi_sort_workspace_size"):
            getattr(L, f).argtypes = [_i64, ctypes.POINTER(sz)]
        L.psi_render_bwd_workspace_size.argtypes = [_i64, _i64, ctypes.c_int, ctypes.POINTER(sz)]
        L.psi_project_surfels.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiCamera), ctypes.c_int,
                                          ctypes.POINTER(PsiRenderOpts), _P, _P, _P, _P]
        L.psi_intersect_tiles.argtypes = [_P, ctypes.POINTER(PsiCamera), ctypes.c_int, ctypes.POINTER(PsiRenderOpts),
                                          _i64, _P, _P, _P, _P, _i64, _P, _P, sz, _P]
        L.psi_sort_keys.argtypes = [_P, _P, _P, _P, _i64, ctypes.c_int, ctypes.c_int, _P, _i64, _P, sz, _P]
        L.psi_sort_keys_noalloc.argtypes = [_P, _P, _P, _P, _i64, ctypes.c_int, ctypes.c_int, _P, _i64, _P]
        L.psi_render_fwd.argtypes = [_P, ctypes.POINTER(PsiFeatures), _P, _P, _P, ctypes.POINTER(PsiCamera),
                                     ctypes.c_int, _i64, ctypes.POINTER(PsiRenderOpts), ctypes.POINTER(PsiFwdOut), _P]
        L.psi_render_bwd.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiFeatures), _P, _P, _P,
                                     ctypes.POINTER(PsiCamera), ctypes.c_int, ctypes.POINTER(PsiRenderOpts), _P, _P, _P,
                                     ctypes.POINTER(PsiFwdOut), ctypes.POINTER(PsiGrads), _P, sz, _P]
        L.psi_ctx_time_kernel.argtypes = [_P, ctypes.c_int, _P, _P]
        L.psi_ctx_set_wait_limit_ns.argtypes = [_P, ctypes.c_uint64]
        L.psi_debug_checks.argtypes = []
        L.psi_quantize_features.argtypes = [_P, _P, _i64, ctypes.c_int, ctypes.c_int, _P, _P, _P]
        L.psi_grads_zero.argtypes = [_P, ctypes.POINTER(PsiGrads), _i64, ctypes.c_int, _P]
        L.psi_tune_render_fwd.argtypes = [_P, ctypes.POINTER(PsiFeatures), _P, _P, _P, ctypes.POINTER(PsiCamera),
                                          ctypes.c_int, _i64, ctypes.POINTER(PsiRenderOpts),
                                          ctypes.POINTER(PsiFwdOut), ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int),
                                          _P]
        L.psi_tune_render_bwd.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiFeatures), _P, _P, _P,
                                          ctypes.POINTER(PsiCamera), ctypes.c_int, ctypes.POINTER(PsiRenderOpts), _P,
                                          _P, _P, ctypes.POINTER(PsiFwdOut), ctypes.POINTER(PsiGrads), _P, sz,
                                          ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int), _P]
        L.psi_ctx_set_render_shape.argtypes = [_P, ctypes.c_int, ctypes.POINTER(PsiRenderOpts), ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int]
        L.psi_ctx_get_render_shape.argtypes = [_P, ctypes.c_int, ctypes.POINTER(PsiRenderOpts), ctypes.c_int,
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.psi_attention_workspace_size.argtypes = [_i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(sz)]
        L.psi_frustum_attention.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiFeatures),
                                            ctypes.POINTER(PsiCamera), ctypes.c_float, _P, ctypes.c_int, _P, _P, _P,
                                            ctypes.c_int, _P, _P, sz, _P]
        L.psi_frustum_attention_bwd.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiFeatures), _P,
                                                ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P,
                                                ctypes.POINTER(PsiGrads), _P, sz, _P]
        L.psi_quat_frames.argtypes = [_P, _P, _i64, _P, _P, _P]
        L.psi_surfel_geometry.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiCamera), _P, ctypes.c_int,
                                          _P]
        L.psi_surfel_geometry_bwd.argtypes = [_P, ctypes.POINTER(PsiSurfels), ctypes.POINTER(PsiCamera), _P,
                                              ctypes.c_int, ctypes.POINTER(PsiGrads), _P]
        L.psi_quat_frames_bwd.argtypes = [_P, _P, _i64, _P, _P, _P, _P]
        L.psi_surfel_regularisers.argtypes = [_P, ctypes.POINTER(PsiSurfels), _P, _P, _P, _i64, ctypes.c_float,
                                               ctypes.c_float, ctypes.c_float, _P, ctypes.POINTER(PsiGrads), _P]
        L.psi_surfel_logits.argtypes = [_P, ctypes.POINTER(PsiFeatures), _i64, _P, ctypes.c_int, _P, ctypes.c_int,
                                         ctypes.c_int, _P]
        L.psi_surfel_labels.argtypes = [_P, ctypes.POINTER(PsiFeatures), _P, _i64, _P, ctypes.c_int, _P, _P, _P,
                                         ctypes.c_int, ctypes.c_int, _P]
        L.psi_decode_queries.argtypes = [_P, _P, _i64, ctypes.c_int, _P, ctypes.c_int, _P, _P, _P, _P]
        _lib = L
    return _lib


def header_symbols(header_path=None):
    """Names of the functions include/psi.h declares (parsed from the header)."""
    import re
    header_path = header_path or os.path.join(os.path.dirname(HERE), "include", "psi.h")
    src = open(header_path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psi_[a-z0-9_]+)\s*\(", src)))


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns a psi_ctx (device status word) on one CUDA device."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        rc = lib().psi_ctx_create(ctypes.byref(h), int(device))
        if rc != PSI_OK:
            raise PsiError(rc, f"psi_ctx_create(device={device}) failed")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            lib().psi_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc, what):
        if rc != PSI_OK:
            raise PsiError(rc, f"{what}: {lib().psi_last_error(self.handle).decode()}")

    def status_fetch(self, stream=None):
        st = _i32(0)
        req = _i64(0)
        self.check(lib().psi_status_fetch(self.handle, _stream(stream), ctypes.byref(st), ctypes.byref(req)),
                   "psi_status_fetch")
        return int(st.value), int(req.value)


def default_opts(**kw) -> PsiRenderOpts:
    o = PsiRenderOpts()
    lib().psi_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def cameras(cams) -> ctypes.Array:
    """Host psi_camera array from scenegen.Camera objects."""
    arr = (PsiCamera * len(cams))()
    for i, c in enumerate(cams):
        a = c.as_array()
        arr[i].R[:] = [float(x) for x in a[:9]]
        arr[i].t[:] = [float(x) for x in a[9:12]]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(x) for x in a[12:16])
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def view_layout(cams_arr, n_views, opts):
    tb = np.zeros(n_views + 1, np.int64)
    pb = np.zeros(n_views + 1, np.int64)
    rc = lib().psi_view_layout(cams_arr, n_views, ctypes.byref(opts), tb.ctypes.data_as(_P), pb.ctypes.data_as(_P))
    if rc != PSI_OK:
        raise PsiError(rc, "psi_view_layout")
    return tb, pb


def _ws(fn, n):
    b = ctypes.c_size_t(0)
    rc = getattr(lib(), fn)(int(n), ctypes.byref(b))
    if rc != PSI_OK:
        raise PsiError(rc, fn)
    return int(b.value)


def intersect_workspace_size(n_records):
    return _ws("psi_intersect_workspace_size", n_records)


def sort_workspace_size(capacity):
    return _ws("psi_sort_workspace_size", capacity)


def render_bwd_workspace_size(n_records, n_pix=0, top_k=0):
    b = ctypes.c_size_t(0)
    rc = lib().psi_render_bwd_workspace_size(int(n_records), int(n_pix), int(top_k), ctypes.byref(b))
    if rc != PSI_OK:
        raise PsiError(rc, "psi_render_bwd_workspace_size")
    return int(b.value)


def surfels_struct(mu, tu, tv, scale, opacity, rgb) -> PsiSurfels:
    return PsiSurfels(_ptr(mu), _ptr(tu), _ptr(tv), _ptr(scale), _ptr(opacity), _ptr(rgb), int(mu.shape[0]))


def features_struct(data, scale, dtype) -> PsiFeatures:
    if data is None:
        return PsiFeatures(None, None, F32, 0)
    return PsiFeatures(_ptr(data), _ptr(scale), int(dtype), int(data.shape[1]))


# ---- entry points (same names as the C ABI) -------------------------------

def psi_project_surfels(ctx, s, cams_arr, n_views, opts, records, bin_records, tiles_touched, stream=None):
    ctx.check(lib().psi_project_surfels(ctx.handle, ctypes.byref(s), cams_arr, n_views, ctypes.byref(opts),
                                        _ptr(records), _ptr(bin_records), _ptr(tiles_touched), _stream(stream)),
              "psi_project_surfels")


def psi_intersect_tiles(ctx, cams_arr, n_views, opts, n_surfels, bin_records, tiles_touched, keys, vals, capacity,
                        d_num_pairs, workspace, stream=None):
    ctx.check(lib().psi_intersect_tiles(ctx.handle, cams_arr, n_views, ctypes.byref(opts), int(n_surfels),
                                        _ptr(bin_records), _ptr(tiles_touched), _ptr(keys), _ptr(vals), int(capacity),
                                        _ptr(d_num_pairs), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                        _stream(stream)), "psi_intersect_tiles")


def psi_sort_keys(ctx, keys, vals, d_num_pairs, capacity, begin_bit, end_bit, tile_ranges, n_tiles_total, workspace,
                  stream=None):
    ctx.check(lib().psi_sort_keys(ctx.handle, _ptr(keys), _ptr(vals), _ptr(d_num_pairs), int(capacity), int(begin_bit),
                                  int(end_bit), _ptr(tile_ranges), int(n_tiles_total), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _stream(stream)), "psi_sort_keys")


def psi_sort_keys_noalloc(ctx, keys, vals, d_num_pairs, capacity, begin_bit, end_bit, tile_ranges, n_tiles_total,
                          stream=None):
    ctx.check(lib().psi_sort_keys_noalloc(ctx.handle, _ptr(keys), _ptr(vals), _ptr(d_num_pairs), int(capacity),
                                          int(begin_bit), int(end_bit), _ptr(tile_ranges), int(n_tiles_total),
                                          _stream(stream)), "psi_sort_keys_noalloc")


def psi_render_fwd(ctx, feats, records, vals, tile_ranges, cams_arr, n_views, n_surfels, opts, out: PsiFwdOut,
                   stream=None):
    ctx.check(lib().psi_render_fwd(ctx.handle, ctypes.byref(feats), _ptr(records), _ptr(vals), _ptr(tile_ranges),
                                   cams_arr, n_views, int(n_surfels), ctypes.byref(opts), ctypes.byref(out),
                                   _stream(stream)), "psi_render_fwd")


def psi_render_bwd(ctx, s, feats, records, vals, tile_ranges, cams_arr, n_views, opts, g_rgb, g_F, g_T,
                   saved, grads: PsiGrads, workspace, stream=None):
    """saved: a PsiFwdOut holding the forward's T, n_last (and topk_ids,
    topk_w when top_k > 0) of this frame, or None to recompute them."""
    ctx.check(lib().psi_render_bwd(ctx.handle, ctypes.byref(s), ctypes.byref(feats), _ptr(records), _ptr(vals),
                                   _ptr(tile_ranges), cams_arr, n_views, ctypes.byref(opts), _ptr(g_rgb), _ptr(g_F),
                                   _ptr(g_T), None if saved is None else ctypes.byref(saved), ctypes.byref(grads),
                                   _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)), "psi_render_bwd")


RENDER_SHAPES = 16


def psi_tune_render_fwd(ctx, feats, records, vals, tile_ranges, cams_arr, n_views, n_surfels, opts, out: PsiFwdOut,
                        reps=3, stream=None):
    """Time every launch shape of the forward compositing kernel on this
    frame, keep the fastest in the context; returns (ms per shape, best)."""
    ms = (ctypes.c_float * RENDER_SHAPES)()
    best = ctypes.c_int(-1)
    ctx.check(lib().psi_tune_render_fwd(ctx.handle, ctypes.byref(feats), _ptr(records), _ptr(vals),
                                        _ptr(tile_ranges), cams_arr, n_views, int(n_surfels), ctypes.byref(opts),
                                        ctypes.byref(out), int(reps), ms, ctypes.byref(best), _stream(stream)),
              "psi_tune_render_fwd")
    return [float(x) for x in ms], int(best.value)


def psi_tune_render_bwd(ctx, s, feats, records, vals, tile_ranges, cams_arr, n_views, opts, g_rgb, g_F, g_T,
                        saved, grads: PsiGrads, workspace, reps=3, stream=None):
    """The same for the adjoint (the gradient buffers are left zeroed)."""
    ms = (ctypes.c_float * RENDER_SHAPES)()
    best = ctypes.c_int(-1)
    ctx.check(lib().psi_tune_render_bwd(ctx.handle, ctypes.byref(s), ctypes.byref(feats), _ptr(records), _ptr(vals),
                                        _ptr(tile_ranges), cams_arr, n_views, ctypes.byref(opts), _ptr(g_rgb),
                                        _ptr(g_F), _ptr(g_T), None if saved is None else ctypes.byref(saved),
                                        ctypes.byref(grads), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), int(reps), ms,
                                        ctypes.byref(best), _stream(stream)), "psi_tune_render_bwd")
    return [float(x) for x in ms], int(best.value)


def psi_ctx_set_render_shape(ctx, which, opts, feat_dtype, saved, shape):
    ctx.check(lib().psi_ctx_set_render_shape(ctx.handle, int(which), ctypes.byref(opts), int(feat_dtype), int(saved),
                                             int(shape)), "psi_ctx_set_render_shape")


def psi_ctx_get_render_shape(ctx, which, opts, feat_dtype, saved):
    v = ctypes.c_int(-1)
    ctx.check(lib().psi_ctx_get_render_shape(ctx.handle, int(which), ctypes.byref(opts), int(feat_dtype), int(saved),
                                             ctypes.byref(v)), "psi_ctx_get_render_shape")
    return int(v.value)


def psi_quantize_features(ctx, f, n, dim, dtype, q, scale=None, stream=None):
    ctx.check(lib().psi_quantize_features(ctx.handle, _ptr(f), int(n), int(dim), int(dtype), _ptr(q), _ptr(scale),
                                          _stream(stream)), "psi_quantize_features")


def psi_grads_zero(ctx, grads: "PsiGrads", n, dim, stream=None):
    ctx.check(lib().psi_grads_zero(ctx.handle, ctypes.byref(grads), int(n), int(dim), _stream(stream)),
              "psi_grads_zero")


def psi_ctx_set_wait_limit_ns(ctx, ns):
    """Limit of the kernels' bounded waits on this context (0 = the default 1 s)."""
    ctx.check(lib().psi_ctx_set_wait_limit_ns(ctx.handle, int(ns)), "psi_ctx_set_wait_limit_ns")


def psi_ctx_time_kernel(ctx, kernel, ev_begin, ev_end):
    """Arm a one-shot pair of timing events (torch.cuda.Event(enable_timing=True),
    already recorded once so that the CUDA event exists) around the next
    eager launch of `kernel` (KERNEL_BWD_FEAT / KERNEL_BWD_WALK)."""
    b = None if ev_begin is None else ctypes.c_void_p(ev_begin.cuda_event)
    e = None if ev_end is None else ctypes.c_void_p(ev_end.cuda_event)
    ctx.check(lib().psi_ctx_time_kernel(ctx.handle, int(kernel), b, e), "psi_ctx_time_kernel")


def attention_workspace_size(n, C, d, n_q):
    b = ctypes.c_size_t(0)
    rc = lib().psi_attention_workspace_size(int(n), int(C), int(d), int(n_q), ctypes.byref(b))
    if rc != PSI_OK:
        raise PsiError(rc, "psi_attention_workspace_size")
    return int(b.value)


def psi_frustum_attention(ctx, s, feats, cam, z_near, Q, n_q, WQ, WK, WV, d, out, workspace, stream=None):
    """cam: one PsiCamera (e.g. cameras([c])[0])."""
    ctx.check(lib().psi_frustum_attention(ctx.handle, ctypes.byref(s), ctypes.byref(feats), ctypes.byref(cam),
                                          float(z_near), _ptr(Q), int(n_q), _ptr(WQ), _ptr(WK), _ptr(WV), int(d),
                                          _ptr(out), _ptr(workspace), workspace.numel() * workspace.element_size(),
                                          _stream(stream)), "psi_frustum_attention")


def psi_frustum_attention_bwd(ctx, s, feats, Q, n_q, WQ, WK, WV, d, g_out, g_Q, g_WQ, g_WK, g_WV,
                              grads: PsiGrads, workspace, stream=None):
    ctx.check(lib().psi_frustum_attention_bwd(ctx.handle, ctypes.byref(s), ctypes.byref(feats), _ptr(Q), int(n_q),
                                              _ptr(WQ), _ptr(WK), _ptr(WV), int(d), _ptr(g_out), _ptr(g_Q), _ptr(g_WQ),
                                              _ptr(g_WK), _ptr(g_WV), ctypes.byref(grads), _ptr(workspace),
                                              workspace.numel() * workspace.element_size(), _stream(stream)),
              "psi_frustum_attention_bwd")


def psi_surfel_geometry(ctx, s, cam_arr, table, ld, stream=None):
    """cam_arr: a one-camera array from cameras([cam])."""
    ctx.check(lib().psi_surfel_geometry(ctx.handle, ctypes.byref(s), cam_arr, _ptr(table), int(ld), _stream(stream)),
              "psi_surfel_geometry")


def psi_surfel_geometry_bwd(ctx, s, cam_arr, g_table, ld, grads: PsiGrads, stream=None):
    ctx.check(lib().psi_surfel_geometry_bwd(ctx.handle, ctypes.byref(s), cam_arr, _ptr(g_table), int(ld),
                                            ctypes.byref(grads), _stream(stream)), "psi_surfel_geometry_bwd")


def psi_quat_frames(ctx, q, n, tu, tv, stream=None):
    ctx.check(lib().psi_quat_frames(ctx.handle, _ptr(q), int(n), _ptr(tu), _ptr(tv), _stream(stream)),
              "psi_quat_frames")


def psi_quat_frames_bwd(ctx, q, n, g_tu, g_tv, g_q, stream=None):
    ctx.check(lib().psi_quat_frames_bwd(ctx.handle, _ptr(q), int(n), _ptr(g_tu), _ptr(g_tv), _ptr(g_q),
                                        _stream(stream)), "psi_quat_frames_bwd")


def psi_surfel_regularisers(ctx, s, node_of, node_mu, node_n, n_nodes, lambda_n, w_geo, w_iso, losses,
                            grads: PsiGrads, stream=None):
    ctx.check(lib().psi_surfel_regularisers(ctx.handle, ctypes.byref(s), _ptr(node_of), _ptr(node_mu), _ptr(node_n),
                                            int(n_nodes), float(lambda_n), float(w_geo), float(w_iso), _ptr(losses),
                                            ctypes.byref(grads), _stream(stream)), "psi_surfel_regularisers")


def psi_surfel_logits(ctx, feats, n, Q, n_q, table, table_dtype, ld, stream=None):
    ctx.check(lib().psi_surfel_logits(ctx.handle, ctypes.byref(feats), int(n), _ptr(Q), int(n_q), _ptr(table),
                                      int(table_dtype), int(ld), _stream(stream)), "psi_surfel_logits")


def psi_surfel_labels(ctx, feats, centres, n, Q, n_q, q_mu, q_cov, labels, labels_dtype, ld, stream=None):
    ctx.check(lib().psi_surfel_labels(ctx.handle, ctypes.byref(feats), _ptr(centres), int(n), _ptr(Q), int(n_q),
                                      _ptr(q_mu), _ptr(q_cov), _ptr(labels), int(labels_dtype), int(ld),
                                      _stream(stream)), "psi_surfel_labels")


def psi_decode_queries(ctx, F, n_pix, D, Q, n_q, T, ids, logits=None, stream=None):
    ctx.check(lib().psi_decode_queries(ctx.handle, _ptr(F), int(n_pix), int(D), _ptr(Q), int(n_q), _ptr(T), _ptr(ids),
                                       _ptr(logits), _stream(stream)), "psi_decode_queries")
