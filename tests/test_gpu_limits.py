"""The path at its documented limits against the oracle (needs a GPU): the
largest feature dimension (256: two float4 chunks per lane in the feature
adjoints), the largest number of views in one launch (64; 65 is refused)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import opts_of
from .test_gpu_grad import _grad_compare
from .test_gpu_parity import _compare_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


@pytest.mark.parametrize("K", [0, 8])
def test_feature_dim_256(ctx, K):
    from paper_2604_10982_gb300 import pipeline as pl
    w = sg.dense_box(n=3000, d=256, width=96, height=64)
    cams = [w.cameras[0]]
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=K > 0)
    scene = pl.DeviceScene(w.surfels, w.features)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=256, want_topk_ids=K > 0)
    r.frame(scene)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    _compare_render(r, scene, w, cams, o, 256, w.features.astype(np.float64))
    _grad_compare(ctx, w, cams, o, 256)


def _views(k):
    return [sg.look_camera((0.05 * i - 1.6, -6.0 - 0.02 * i, 1.5), 0.01 * i - 0.3, 24 + i % 9, 16 + i % 7,
                           20.0 + i) for i in range(k)]


def test_max_views_one_launch(ctx):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=3000, d=16)
    cams = _views(64)
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
    scene = pl.DeviceScene(w.surfels, w.features)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=16)
    r.frame(scene)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    assert r.n_tiles == sum(((c.width + 15) // 16) * ((c.height + 15) // 16) for c in cams)
    _compare_render(r, scene, w, cams, o, 16, w.features.astype(np.float64))
    with pytest.raises(psi.PsiError) as e:
        pl.make_renderer(ctx, scene, _views(65), opts_of(o), D=16)
    assert e.value.code == psi.PSI_ERR_INVALID_ARG
