"""Depth and normal maps of the 2D-surfel model on the GPU against the oracle:
the per-surfel geometry table, its blending by the dense feature path, and
its adjoint (needs a GPU)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import flags, opts_of
from .test_gpu_grad import _grad_compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


@pytest.fixture(scope="module")
def box():
    return sg.dense_box(n=6000, d=16)


def _table(ctx, w, cam, ld=16):
    from paper_2604_10982_gb300 import pipeline as pl
    scene = pl.DeviceScene(w.surfels, None)
    T = pl.surfel_geometry(ctx, scene, cam, ld=ld)
    torch.cuda.synchronize()
    return scene, T


@pytest.mark.parametrize("ld", [16, 32])
def test_geometry_table_matches_oracle(ctx, box, ld):
    cam = box.cameras[0]
    _, T = _table(ctx, box, cam, ld)
    g = T.cpu().numpy().astype(np.float64)
    ref = orc.surfel_geometry(box.surfels, cam)
    assert np.all(g[:, 4:] == 0)
    assert np.abs(g[:, 0] - ref[:, 0]).max() <= 1e-6 * np.abs(ref[:, 0]).max()
    assert np.abs(g[:, 1:4] - ref[:, 1:4]).max() < 1e-5


def test_depth_normal_maps_blend_like_features(ctx, box):
    """The table as a dense float32 feature table: the GPU maps against the
    oracle's FP64 blend of the same stored table."""
    from paper_2604_10982_gb300 import pipeline as pl
    cam = box.cameras[0]
    scene, T = _table(ctx, box, cam)
    gs = pl.label_scene(scene, T)
    o = orc.Opts(mode=orc.EXACT, top_k=0)
    r = pl.make_renderer(ctx, gs, [cam], opts_of(o), D=16)
    r.frame(gs)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    # the feature bar 1e-4 * max(1, max|f|) (depths reach ~10 m), RGB and T at 1e-4
    T64 = T.cpu().numpy().astype(np.float64)
    ref = orc.render(box.surfels, cam, o, feat=T64)
    st, ic, _ = flags(ref, cam)
    ok = ~(st | ic)
    assert ok.mean() > 0.98
    e_F = np.abs(r.F.cpu().numpy().astype(np.float64) - ref["F"]).max(1)
    assert e_F[ok].max() <= 1e-4 * max(1.0, np.abs(T64).max()), e_F[ok].max()
    assert np.abs(r.T.cpu().numpy() - ref["T"])[ok].max() < 1e-4
    # a covered pixel's depth map divided by its coverage lies within the surfels' depth range
    F = r.F.cpu().numpy()
    cov = 1.0 - r.T.cpu().numpy()
    m = cov > 0.5
    d = F[m, 0] / cov[m]
    z = T[:, 0].cpu().numpy()
    assert m.sum() > 1000 and d.min() >= z.min() - 1e-3 and d.max() <= z.max() + 1e-3


def test_geometry_adjoint_matches_oracle(ctx, box):
    from paper_2604_10982_gb300 import psi
    cam = box.cameras[0]
    scene, _ = _table(ctx, box, cam)
    n = box.surfels.n
    g = sg.make_upstream(16 * n, 5, 0).reshape(n, 16).astype(np.float32)
    gt = torch.from_numpy(g).cuda()
    grads = {k: torch.zeros(n, 3, device="cuda") for k in ("mu", "tu", "tv")}
    gs = psi.PsiGrads(psi._ptr(grads["mu"]), psi._ptr(grads["tu"]), psi._ptr(grads["tv"]), None, None, None, None)
    psi.psi_surfel_geometry_bwd(ctx, scene.surfels_struct(), psi.cameras([cam]), gt, 16, gs)
    torch.cuda.synchronize()
    ref = orc.surfel_geometry_grad(box.surfels, cam, g[:, :4].astype(np.float64))
    for k in ("mu", "tu", "tv"):
        a = grads[k].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - ref[k]) <= 1e-5 * np.linalg.norm(ref[k]), k


def test_rendered_geometry_gradients(ctx):
    """Both adjoint forms of the render of the table (dense, EXACT) against the
    oracle, the table's gradient included; the table's own adjoint is pinned
    above, so the chain to mu, t_u, t_v is covered."""
    w = sg.crop_scene(n=500, d=16, size=64)
    cam = w.cameras[0]
    _, T = _table(ctx, w, cam)
    w2 = dataclasses.replace(w, features=T.cpu().numpy())
    _grad_compare(ctx, w2, [cam], orc.Opts(mode=orc.EXACT, top_k=0), 16)
