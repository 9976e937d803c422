"""Failure detection on the GPU (needs a GPU): the kernels' bounded waits give
up without faulting or hanging. With the context's wait limit cut to 1 ns the
compositing kernel (and, when its waits run out, the query decode) raises
PSI_ERR_TIMEOUT with its wait site, returns, writes nothing outside its
outputs, and leaves the context usable: with the default limit restored the
next frame matches the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import check_values, multi_cams, opts_of

pytestmark = pytest.mark.gpu

SENT = -7.0
G = 4096  # guard elements on both sides of every output


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    c = psi.Context(0)
    yield c
    psi.psi_ctx_set_wait_limit_ns(c, 0)


def _guarded(n, dtype, fill):
    big = torch.full((n + 2 * G,), fill, dtype=dtype, device="cuda")
    return big, big[G:G + n]


def _guards_intact(big, fill):
    return bool((big[:G] == fill).all()) and bool((big[-G:] == fill).all())


def test_wait_limit_timeout_then_clean_frame(ctx):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=6000, d=64)
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=64, F_dtype=psi.BF16)
    P, K = r.n_pix, 8
    rgb_b, rgb = _guarded(3 * P, torch.float32, SENT)
    T_b, T = _guarded(P, torch.float32, SENT)
    nl_b, nl = _guarded(P, torch.int32, -7)
    F_b, F = _guarded(P * 64, torch.bfloat16, SENT)
    id_b, ids = _guarded(P * K, torch.int32, -7)
    w_b, tw = _guarded(P * K, torch.float32, SENT)
    r.rgb, r.T, r.n_last, r.F = rgb.view(3, P), T, nl, F.view(P, 64)
    r.topk_ids, r.topk_w = ids.view(P, K), tw.view(P, K)
    bigs = [(rgb_b, SENT), (T_b, SENT), (nl_b, -7), (F_b, SENT), (id_b, -7), (w_b, SENT)]
    Q = torch.from_numpy(sg.make_queries(40, 64, 3)).cuda().to(torch.bfloat16)
    dec_b, dec = _guarded(P, torch.int32, -7)

    r.project(scene)
    r.intersect()
    r.sort()
    assert ctx.status_fetch() == (0, 0)
    psi.psi_ctx_set_wait_limit_ns(ctx, 1)
    r.render(scene)
    st, site = ctx.status_fetch()
    assert st == psi.PSI_ERR_TIMEOUT and site == 1, (st, site)
    psi.psi_decode_queries(ctx, r.F, P, 64, Q, 40, r.T, dec)
    st, site = ctx.status_fetch()
    assert st in (0, psi.PSI_ERR_TIMEOUT) and (st == 0 or site in (4, 5, 6)), (st, site)
    torch.cuda.synchronize()
    assert all(_guards_intact(b, f) for b, f in bigs) and _guards_intact(dec_b, -7)

    with pytest.raises(psi.PsiError):
        psi.psi_ctx_set_wait_limit_ns(ctx, 10**11)
    psi.psi_ctx_set_wait_limit_ns(ctx, 0)
    r.render(scene)
    psi.psi_decode_queries(ctx, r.F, P, 64, Q, 40, r.T, dec)
    assert ctx.status_fetch() == (0, 0)
    assert all(_guards_intact(b, f) for b, f in bigs) and _guards_intact(dec_b, -7)
    deq = pl.dequantize(scene.q, None, psi.BF16)
    rgb_h = r.rgb.cpu().numpy().astype(np.float64)
    T_h = r.T.cpu().numpy().astype(np.float64)
    F_h = r.F.float().cpu().numpy().astype(np.float64)
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        ref = orc.render(w.surfels, cam, o, feat=deq)
        check_values(rgb_h[:, a:b].T, T_h[a:b], F_h[a:b], ref, cam, bf16_rel=2e-2, fmax=np.abs(deq).max())
    rid, L, gap = orc.decode(F_h, Q.float().cpu().numpy().astype(np.float64), T_h)
    tie = gap < 1e-4 * (np.abs(L).max(1) + 1e-6)
    assert ((dec.cpu().numpy() != rid) & ~tie).sum() == 0
