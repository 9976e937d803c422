"""Per-surfel instance labels (Sec. 4.1, Eqs. 4-7) and the rendered identity
(Eq. 8) against the oracle (needs a GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import flags, multi_cams, opts_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _case(n_q, d, n=5000, seed=11):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=n, d=d)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16)
    qf = sg.make_queries(n_q, d, seed) * 4.0
    mu, cov = sg.make_query_gaussians(n_q, seed, (-4, -5, 0), (4, 5, 10))
    Qb = torch.from_numpy(qf).to(torch.bfloat16)
    return w, scene, Qb, mu, cov


def _oracle_labels(w, scene, Qb, mu, cov):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    f = pl.dequantize(scene.q, None, psi.BF16)
    return orc.surfel_labels(f, Qb.float().numpy().astype(np.float64), mu, cov, w.surfels.mu)


@pytest.mark.parametrize("n_q,d", [(7, 64), (100, 128), (128, 128)])
def test_labels_match_oracle(ctx, n_q, d):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w, scene, Qb, mu, cov = _case(n_q, d)
    ref = _oracle_labels(w, scene, Qb, mu, cov)
    L32 = pl.surfel_labels(ctx, scene, Qb, mu, cov, dtype=psi.F32)
    L16 = pl.surfel_labels(ctx, scene, Qb, mu, cov, dtype=psi.BF16)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    ld = L32.shape[1]
    assert ld % 16 == 0 and ld >= n_q
    g32 = L32.cpu().numpy().astype(np.float64)
    g16 = L16.float().cpu().numpy().astype(np.float64)
    assert np.all(g32[:, n_q:] == 0) and np.all(g16[:, n_q:] == 0)
    # FP32 epilogue (fast exponentials) on BF16 products accumulated in FP32
    assert np.abs(g32[:, :n_q] - ref).max() < 2e-5
    assert np.abs(g16[:, :n_q] - ref).max() < 4e-3
    assert np.allclose(g32[:, :n_q].sum(1), 1.0, atol=1e-5)


def test_labels_single_query_and_errors(ctx):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w, scene, Qb, mu, cov = _case(1, 64, n=700)
    L = pl.surfel_labels(ctx, scene, Qb, mu, cov, dtype=psi.F32)
    torch.cuda.synchronize()
    g = L.cpu().numpy()
    assert np.all(g[:, 0] == 1.0) and np.all(g[:, 1:] == 0.0)
    # FP8 storage is not supported by the tensor-core path; ld must be a multiple of 16
    s8 = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.FP8_E4M3)
    with pytest.raises(psi.PsiError) as e:
        pl.surfel_labels(ctx, s8, Qb, mu, cov)
    assert e.value.code == psi.PSI_ERR_UNSUPPORTED
    with pytest.raises(psi.PsiError) as e:
        pl.surfel_labels(ctx, scene, Qb, mu, cov, ld=24)
    assert e.value.code == psi.PSI_ERR_INVALID_ARG


def test_rendered_identity(ctx):
    """Eq. 8: the label table rendered with Top-K selection; the fused
    per-pixel argmax (no feature map written) against the oracle's argmax of
    the blended labels. Near ties and excused pixels are counted, not
    compared."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w, scene, Qb, mu, cov = _case(100, 128, n=6000)
    L = pl.surfel_labels(ctx, scene, Qb, mu, cov, dtype=psi.BF16)
    ls = pl.label_scene(scene, L)
    cams = multi_cams()[:2]
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
    r = pl.make_renderer(ctx, ls, cams, opts_of(o), D=ls.D, F_dtype=psi.F32)
    r.frame(ls, want_F=False)
    r.render(ls, want_F=False, argmax=True)
    ids_nof = r.argmax.clone()
    r.render(ls, want_F=True, argmax=True)  # the same ids when F is also written
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    assert torch.equal(ids_nof, r.argmax)
    lab = L.float().cpu().numpy().astype(np.float64)  # the stored label values
    gids = r.argmax.cpu().numpy()
    F = r.F.cpu().numpy()
    compared = 0
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        ref = orc.render(w.surfels, cam, o, feat=lab)
        rid, gap = orc.label_ids(ref["F"], ref["T"])
        st, ic, nt = flags(ref, cam)
        ok = ~(st | ic | nt) & ((gap > 1e-4) | (rid == -1))
        assert np.array_equal(gids[a:b][ok], rid[ok])
        # the ids are the argmax of the GPU's own FP32 mixture as well
        own = np.where((1.0 - r.T.cpu().numpy()[a:b]) < 1e-4, -1, np.argmax(F[a:b], axis=1))
        tie = (-np.sort(-F[a:b], axis=1))
        sure = (tie[:, 0] - tie[:, 1]) > 1e-6
        assert np.array_equal(gids[a:b][sure], own[sure])
        compared += int(ok.sum())
    assert compared > 0.5 * sum(c.width * c.height for c in cams)


def test_fused_decode_through_logit_table(ctx):
    """The decode fused into compositing: per-surfel logits f_q^T f_g rendered
    with the Top-K weights and the fused argmax give the decode's ids (a6)
    without a feature map; compared with the FP64 oracle's decode of the
    oracle's own feature map and with the tensor-core decode of the GPU's F."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w, scene, Qb, mu, cov = _case(100, 128, n=6000)
    T = pl.surfel_logits(ctx, scene, Qb, dtype=psi.F32)
    torch.cuda.synchronize()
    f = pl.dequantize(scene.q, None, psi.BF16)
    qf = Qb.float().numpy().astype(np.float64)
    ref_tab = f @ qf.T
    tab = T.cpu().numpy().astype(np.float64)
    assert np.all(tab[:, 100:] == 0)
    assert np.abs(tab[:, :100] - ref_tab).max() <= 1e-5 * max(1.0, np.abs(ref_tab).max())
    cams = multi_cams()[:2]
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
    ts = pl.label_scene(scene, T)
    r = pl.make_renderer(ctx, ts, cams, opts_of(o), D=ts.D)
    r.frame(ts, want_F=False)
    r.render(ts, want_F=False, argmax=True)
    ids_fused = r.argmax.cpu().numpy()
    # the unfused path: features rendered to F (BF16), then the tensor-core decode
    rf = pl.make_renderer(ctx, scene, cams, opts_of(o), D=128, F_dtype=psi.BF16)
    rf.frame(scene)
    ids_dec = torch.empty(rf.n_pix, dtype=torch.int32, device="cuda")
    psi.psi_decode_queries(ctx, rf.F, rf.n_pix, 128, Qb.cuda(), 100, rf.T, ids_dec)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    ids_dec = ids_dec.cpu().numpy()
    compared = 0
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        ref = orc.render(w.surfels, cam, o, feat=f)
        rid, L, gap = orc.decode(ref["F"], qf, ref["T"])
        st, ic, nt = flags(ref, cam)
        ok = ~(st | ic | nt) & ((gap > 1e-3 * (np.abs(L).max(1) + 1e-6)) | (rid == -1))
        assert np.array_equal(ids_fused[a:b][ok], rid[ok])
        # the unfused decode rounds F to BF16 first: equal wherever the margin is clear
        clear = ok & (gap > 2e-2 * (np.abs(L).max(1) + 1e-6))
        assert np.array_equal(ids_fused[a:b][clear], ids_dec[a:b][clear])
        compared += int(ok.sum())
    assert compared > 0.5 * sum(c.width * c.height for c in cams)
