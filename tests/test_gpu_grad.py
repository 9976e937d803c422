"""Hand-written adjoint vs the oracle's FP64 gradient (needs a GPU).

Upstream gradients are zeroed on pixels the forward comparison excuses
(threshold straddles, near ties, ill-conditioned), on both sides, so the
comparison is exact apart from float32 rounding: the gradient is linear in
the upstream gradient."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import flags, multi_cams, opts_of

pytestmark = pytest.mark.gpu

KEYS = ("mu", "tu", "tv", "scale", "opacity", "rgb", "feat")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _upstream(cams, D, seed, pixel_mask=None):
    P = sum(c.width * c.height for c in cams)
    gC = sg.make_upstream(3 * P, seed, 0).reshape(3, P)
    gF = sg.make_upstream(D * P, seed, 1).reshape(P, D) if D else None
    gT = sg.make_upstream(P, seed, 2)
    if pixel_mask is not None:
        gC = gC * pixel_mask[None, :]
        gT = gT * pixel_mask
        if gF is not None:
            gF = gF * pixel_mask[:, None]
    return gC, gF, gT


def _grad_compare(ctx, w, cams, o, D, tol=1e-3, sample_pixels=None, feat_dtype=None):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    fdt = psi.F32 if feat_dtype is None else feat_dtype
    scene = pl.DeviceScene(w.surfels, w.features if D else None, feat_dtype=fdt)
    if D and fdt != psi.F32:
        # the oracle sees the stored (dequantised) feature values
        w = dataclasses.replace(w, features=pl.dequantize(scene.q, scene.qscale, fdt))
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=D)
    r.frame(scene)
    # excusal mask from the oracle's forward diagnostics, evaluated only on the
    # pixels that carry upstream gradient (all, or a sample)
    P = int(r.pix_base[-1])
    mask = np.zeros(P, np.float32)
    cand = np.arange(P) if sample_pixels is None else np.asarray(sample_pixels)
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        idx = cand[(cand >= a) & (cand < b)] - a
        if len(idx) == 0:
            continue
        ref = orc.render(w.surfels, cam, o, feat=w.features if D else None, pixels=orc.all_pixels(cam)[idx])
        st, ic, nt = flags(ref, cam)
        mask[a + idx] = (~(st | ic | nt)).astype(np.float32)
    gC, gF, gT = _upstream(cams, D, 3, mask)
    tgC = torch.from_numpy(np.ascontiguousarray(gC)).cuda()
    tgF = torch.from_numpy(np.ascontiguousarray(gF)).cuda() if D else None
    tgT = torch.from_numpy(gT).cuda()
    # both adjoint forms: the forward's saved T / last / Top-K ids, and the
    # recomputing walk; each against the oracle, and against each other
    g = r.backward(scene, tgC, tgF, tgT)
    g_re = r.backward(scene, tgC, tgF, tgT, recompute=True)
    torch.cuda.synchronize()
    st, _ = ctx.status_fetch()
    assert st == 0
    # oracle gradient, summed over views
    ref = {k: 0.0 for k in KEYS}
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        sel = np.nonzero(mask[a:b])[0]
        pix = orc.all_pixels(cam)[sel]
        gv = orc.render_grad(w.surfels, cam, o, gC[:, a:b].T[sel], feat=w.features if D else None,
                             gF=gF[a:b][sel] if D else None, gT=gT[a:b][sel], pixels=pix)
        for k in KEYS:
            ref[k] = ref[k] + gv[k]
    report = {}
    for k in KEYS:
        if k == "feat" and not D:
            continue
        den = np.linalg.norm(ref[k])
        assert den > 0, k
        for form, gg in (("saved", g), ("recompute", g_re)):
            gk = gg[k].cpu().numpy().astype(np.float64).reshape(ref[k].shape)
            rel = np.linalg.norm(gk - ref[k]) / max(den, 1e-30)
            report[(k, form)] = rel
            assert rel < tol, (k, form, rel)
        # same arithmetic; only the order of the float32 atomic additions differs
        a, b = g[k].double(), g_re[k].double()
        assert torch.linalg.norm(a - b).item() <= 1e-5 * max(torch.linalg.norm(a).item(), 1e-30), k
    return report


def test_grad_crop_topk(ctx):
    w = sg.crop_scene(n=500, d=32, size=64)
    o = orc.Opts(mode=orc.EXACT, top_k=16)
    rep = _grad_compare(ctx, w, w.cameras, o, 32)
    print(rep)


def test_grad_crop_dense(ctx):
    w = sg.crop_scene(n=500, d=32, size=64)
    o = orc.Opts(mode=orc.AABB, top_k=0)
    _grad_compare(ctx, w, w.cameras, o, 32)


@pytest.mark.parametrize("K", [1, 8])
def test_grad_box_multiview(ctx, K):
    w = sg.dense_box(n=4000, d=16)
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=True)
    _grad_compare(ctx, w, multi_cams(), o, 16)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_grad_quantised_features_d128(ctx, dtype):
    """The bench's feature form: D=128 stored in BF16 (32-byte row loads) or
    FP8-E4M3 with per-channel scales, K=8, EXACT + opacity radius."""
    from paper_2604_10982_gb300 import psi
    w = sg.dense_box(n=3000, d=128)
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
    _grad_compare(ctx, w, multi_cams()[:2], o, 128, feat_dtype=psi.BF16 if dtype == "bf16" else psi.FP8_E4M3)


@pytest.mark.parametrize("K,D,dtype", [(16, 64, "bf16"), (8, 256, "bf16"), (32, 48, "fp8")])
def test_grad_feature_kernel_forms(ctx, K, D, dtype):
    """The feature adjoint outside its register-resident form (K > 8 or
    D > 128: every selecting pixel's g_F row read per surfel, two channel
    chunks per lane at D = 256), against the oracle."""
    from paper_2604_10982_gb300 import psi
    w = sg.dense_box(n=3000, d=D)
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=True)
    _grad_compare(ctx, w, multi_cams()[:2], o, D, feat_dtype=psi.BF16 if dtype == "bf16" else psi.FP8_E4M3)


def test_grad_rgb_only(ctx):
    w = sg.dense_box(n=3000, d=16)
    o = orc.Opts(mode=orc.SPHERE, top_k=0)
    _grad_compare(ctx, w, multi_cams()[:1], o, 0)


def test_grad_full_size_sampled_pixels(ctx):
    """960x540, 500k surfels, D=128, K=16: upstream gradient on 48 sampled
    pixels, full gradient vectors compared."""
    w = sg.grad_scene()
    cam = w.cameras[0]
    rng = np.random.default_rng(1)
    pix = rng.choice(cam.width * cam.height, 48, replace=False)
    o = orc.Opts(mode=orc.EXACT, top_k=16)
    _grad_compare(ctx, w, w.cameras, o, 128, sample_pixels=pix)


def test_autograd_function(ctx):
    from paper_2604_10982_gb300 import pipeline as pl
    w = sg.crop_scene(n=300, d=16, size=48)
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene = pl.DeviceScene(w.surfels, w.features)
    for t in (scene.mu, scene.tu, scene.tv, scene.scale, scene.opacity, scene.rgb, scene.q):
        t.requires_grad_(True)
    r = pl.make_renderer(ctx, scene, w.cameras, opts_of(o), D=16)
    rgb, F, T = pl.render_autograd(r, scene)
    loss = (rgb * 0.3).sum() + (F * 0.1).sum() - T.sum()
    loss.backward()
    g = r.backward(scene, torch.full_like(rgb, 0.3), torch.full_like(F, 0.1), torch.full_like(T, -1.0))
    torch.cuda.synchronize()
    assert torch.allclose(scene.mu.grad, g["mu"], rtol=1e-4, atol=1e-6)
    assert torch.allclose(scene.q.grad, g["feat"], rtol=1e-4, atol=1e-6)
    assert float(scene.opacity.grad.abs().sum()) > 0


def test_grad_long_lists_early_exit(ctx):
    """Tile lists spanning many 256-record batches with early termination:
    exercises the adjoint's batch staging in both directions."""
    w = sg.dense_box(n=20000, d=16, width=64, height=48, scale_median=0.25)
    o = orc.Opts(mode=orc.AABB, top_k=8)
    _grad_compare(ctx, w, w.cameras, o, 16)


def test_saved_state_needs_topk_ids(ctx):
    """Saved forward state without the Top-K ids and weights (K > 0) is refused."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.crop_scene(n=200, d=16, size=32)
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene = pl.DeviceScene(w.surfels, w.features)
    r = pl.make_renderer(ctx, scene, w.cameras, opts_of(o), D=16, want_topk_ids=False)
    r.frame(scene)
    assert r.saved_state() is None
    saved = psi.PsiFwdOut(psi._ptr(r.rgb), psi._ptr(r.T), psi._ptr(r.n_last), None, psi.F32, None, None)
    gC = torch.zeros(3, r.n_pix, device="cuda")
    grads = {k: torch.zeros(r.n, 3, device="cuda") for k in ("mu", "tu", "tv", "rgb")}
    gs = psi.PsiGrads(*(psi._ptr(grads.get(k)) for k in ("mu", "tu", "tv", "scale", "opacity", "rgb", "feat")))
    ws = torch.empty(psi.render_bwd_workspace_size(r.n, r.n_pix, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(psi.PsiError) as e:
        psi.psi_render_bwd(ctx, scene.surfels_struct(), scene.features_struct(), r.records, r.vals, r.ranges,
                           r.cams, r.V, r.opts, gC, None, None, saved, gs, ws)
    assert e.value.code == psi.PSI_ERR_INVALID_ARG
    # the recomputing form still runs on the same renderer
    g = r.backward(scene, gC)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0


def test_kernel_timing_events(ctx):
    """psi_ctx_time_kernel brackets the adjoint's feature kernel and list walk
    of the next eager call, once."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.crop_scene(n=300, d=16, size=48)
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene = pl.DeviceScene(w.surfels, w.features)
    r = pl.make_renderer(ctx, scene, w.cameras, opts_of(o), D=16)
    r.frame(scene)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev:
        e.record()
    torch.cuda.synchronize()
    psi.psi_ctx_time_kernel(ctx, psi.KERNEL_BWD_FEAT, ev[0], ev[1])
    psi.psi_ctx_time_kernel(ctx, psi.KERNEL_BWD_WALK, ev[2], ev[3])
    gC = torch.ones(3, r.n_pix, device="cuda")
    gF = torch.ones(r.n_pix, 16, device="cuda")
    r.backward(scene, gC, gF)
    torch.cuda.synchronize()
    t_feat, t_walk = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    assert t_feat > 0 and t_walk > 0
    # disarmed after one call: the events keep their timestamps
    r.backward(scene, gC, gF)
    torch.cuda.synchronize()
    assert ev[2].elapsed_time(ev[3]) == t_walk
    with pytest.raises(psi.PsiError):
        psi.psi_ctx_time_kernel(ctx, 7, ev[0], ev[1])
    with pytest.raises(psi.PsiError):
        psi.psi_ctx_time_kernel(ctx, psi.KERNEL_BWD_WALK, ev[0], None)
