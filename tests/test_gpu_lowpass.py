"""The 2DGS object-space low-pass filter on the GPU against the oracle: binning
and keys bit for bit, renders and both adjoint forms within the parity bar
(needs a GPU). The scenes use surfels of about a pixel, so that the filter's
screen-space term and the surfel's own Gaussian both win somewhere."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import multi_cams, opts_of
from .test_gpu_grad import _grad_compare
from .test_gpu_parity import _compare_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


@pytest.fixture(scope="module")
def small():
    return sg.dense_box(n=6000, d=32, scale_median=0.05)


def _renderer(ctx, w, cams, o, D=0, topk_ids=False):
    from paper_2604_10982_gb300 import pipeline as pl
    scene = pl.DeviceScene(w.surfels, w.features if D else None)
    return scene, pl.make_renderer(ctx, scene, cams, opts_of(o), D=D, want_topk_ids=topk_ids)


@pytest.mark.parametrize("mode", [orc.SPHERE, orc.AABB, orc.EXACT])
@pytest.mark.parametrize("oprad", [False, True])
def test_lowpass_binning_and_keys_bitexact(ctx, small, mode, oprad):
    cams = multi_cams()
    o = orc.Opts(mode=mode, opacity_radius=oprad, lowpass=True)
    scene, r = _renderer(ctx, small, cams, o)
    r.project(scene)
    r.intersect()
    torch.cuda.synchronize()
    n = small.surfels.n
    counts = r.counts.cpu().numpy().view(np.uint32)
    bins = r.bins.cpu().numpy()[: len(cams) * n * 48].view(np.uint32).reshape(len(cams) * n, 12)
    for v, cam in enumerate(cams):
        b = orc.bin_view(small.surfels, cam, o)
        plain = orc.bin_view(small.surfels, cam, orc.Opts(mode=mode, opacity_radius=oprad))
        assert np.array_equal(counts[v * n:(v + 1) * n], b["count"]), v
        # the filter only adds tiles
        assert (b["count"] >= plain["count"]).all() and b["count"].sum() > plain["count"].sum()
        vis = b["count"] > 0
        g = bins[v * n:(v + 1) * n][vis]
        rect = b["rect"][vis].astype(np.uint32)
        assert np.array_equal(g[:, 6], rect[:, 0] | (rect[:, 1] << 16))
        assert np.array_equal(g[:, 7], rect[:, 2] | (rect[:, 3] << 16))
        assert np.array_equal(g[:, 5], b["depth_bits"][vis])
    P = int(r.num_pairs.item())
    ek, ev = orc.emit_pairs(small.surfels, cams, o)
    assert P == len(ek)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), ev)
    r.sort()
    torch.cuda.synchronize()
    sk, sv = orc.sort_pairs(ek, ev)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), sk)
    assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), sv)
    assert ctx.status_fetch()[0] == 0


@pytest.mark.parametrize("K", [0, 8, 32])
def test_lowpass_render(ctx, small, K):
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=K != 0, lowpass=True)
    scene, r = _renderer(ctx, small, cams, o, D=32, topk_ids=K > 0)
    r.frame(scene)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    _compare_render(r, scene, small, cams, o, 32, small.features.astype(np.float64))
    # the filter is active: the same frame without it differs
    o2 = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=K != 0)
    scene2, r2 = _renderer(ctx, small, cams, o2, D=32)
    r2.frame(scene2)
    torch.cuda.synchronize()
    assert (r.T != r2.T).float().mean().item() > 0.05


def test_lowpass_grad_crop(ctx):
    w = sg.crop_scene(n=500, d=32, size=64, scale_median=0.08)
    o = orc.Opts(mode=orc.EXACT, top_k=16, lowpass=True)
    _grad_compare(ctx, w, w.cameras, o, 32)


@pytest.mark.parametrize("K", [0, 8])
def test_lowpass_grad_box_multiview(ctx, K):
    w = sg.dense_box(n=4000, d=16, scale_median=0.05)
    o = orc.Opts(mode=orc.EXACT if K else orc.AABB, top_k=K, opacity_radius=K > 0, lowpass=True)
    _grad_compare(ctx, w, multi_cams(), o, 16)
