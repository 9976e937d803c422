"""16x8 tiles (needs a GPU): the alternative tile shape of the compositing
launch. Binning with 8-row tiles is compared bit for bit with the oracle's
pinned float32 path (its tile size is a parameter), the frame and both adjoint
forms against the FP64 oracle under the same bars as the 16x16 tiles, and the
two tile shapes against each other."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import check_values, multi_cams, opts_of
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
    return sg.dense_box(n=6000, d=32)


@pytest.mark.parametrize("mode", [orc.SPHERE, orc.AABB, orc.EXACT])
def test_tile16x8_keys_sort_bitexact(ctx, box, mode):
    from paper_2604_10982_gb300 import pipeline as pl
    cams = multi_cams()
    o = orc.Opts(mode=mode, top_k=8, opacity_radius=(mode == orc.EXACT), tile_h=8)
    scene = pl.DeviceScene(box.surfels, None)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o))
    r.project(scene)
    r.intersect()
    torch.cuda.synchronize()
    n = box.surfels.n
    counts = r.counts.cpu().numpy().view(np.uint32)
    for v, cam in enumerate(cams):
        b = orc.bin_view(box.surfels, cam, o)
        assert np.array_equal(counts[v * n:(v + 1) * n], b["count"]), v
    P = int(r.num_pairs.item())
    ek, ev = orc.emit_pairs(box.surfels, cams, o)
    assert P == len(ek)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), ev)
    r.sort()
    torch.cuda.synchronize()
    sk, sv = orc.sort_pairs(ek, ev)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), sk)
    assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), sv)
    rg = r.ranges.cpu().numpy().view(np.uint32)[: 2 * r.n_tiles].reshape(-1, 2).astype(np.int64)
    ro = orc.tile_ranges(sk, r.n_tiles).astype(np.int64)
    assert np.array_equal(rg[:, 1] - rg[:, 0], ro[:, 1] - ro[:, 0])
    assert ctx.status_fetch()[0] == 0


@pytest.mark.parametrize("K", [1, 8])
def test_tile16x8_render_matches_oracle(ctx, box, K):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=True, tile_h=8)
    scene = pl.DeviceScene(box.surfels, box.features, feat_dtype=psi.BF16)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=32)
    r.frame(scene)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    feat = pl.dequantize(scene.q, None, psi.BF16)
    rgb = r.rgb.cpu().numpy().astype(np.float64)
    T = r.T.cpu().numpy().astype(np.float64)
    F = r.F.cpu().numpy().astype(np.float64)
    ids = r.topk_ids.cpu().numpy()
    from .gpu_common import flags
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        ref = orc.render(box.surfels, cam, o, feat=feat)
        check_values(rgb[:, a:b].T, T[a:b], F[a:b], ref, cam, fmax=np.abs(feat).max())
        st, ic, nt = flags(ref, cam)
        ok = ~(st | ic | nt)
        same = np.array([set(ids[a + p][ids[a + p] >= 0]) == set(ref["topk"][p][ref["topk"][p] >= 0])
                         for p in range(b - a)])
        assert (ok & ~same).sum() == 0, v
    # against the 16x16 tiles: a 16x8 tile evaluates its pixels with the
    # 16x16 tile's float32 sequence, so the frame is the same bit for bit
    # (n_last, a position in the tile's list, differs with the lists)
    o16 = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=True)
    r16 = pl.make_renderer(ctx, scene, cams, opts_of(o16), D=32)
    r16.frame(scene)
    torch.cuda.synchronize()
    for name in ("rgb", "T", "F", "topk_ids", "topk_w"):
        assert torch.equal(getattr(r, name), getattr(r16, name)), name


def test_tile16x8_gradients_match_oracle(ctx):
    w = sg.dense_box(n=4000, d=16)
    o = orc.Opts(mode=orc.EXACT, top_k=8, tile_h=8)
    _grad_compare(ctx, w, multi_cams(), o, 16)


def test_tile16x8_rejects_dense_and_lowpass(ctx, box):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    cams = multi_cams()[:1]
    scene = pl.DeviceScene(box.surfels, None)
    for kw in (dict(top_k=0), dict(top_k=8, lowpass=True), dict(top_k=16)):
        o = orc.Opts(mode=orc.EXACT, tile_h=8, **kw)
        with pytest.raises(psi.PsiError):
            r = pl.Renderer(ctx, scene.n, cams, opts_of(o), 1024)
            r.project(scene)


def test_tile16x8_paired_walk_equals_single(ctx):
    """16x8 tiles with the adjoint's paired walk (launch shape bit 3, two
    pixel warps of 8x8 blocks per tile), alone and persistent: the same
    gradients as the one-pixel walk up to the order of float32 atomics."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=4000, d=32)
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True, tile_h=8)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=32)
    r.frame(scene)
    P = r.n_pix
    g = torch.Generator(device="cpu").manual_seed(7)
    gC, gF, gT = torch.randn(3, P, generator=g).cuda(), torch.randn(P, 32, generator=g).cuda(), torch.randn(P, generator=g).cuda()
    out = {}
    for shape in (0, 8, 12):
        psi.psi_ctx_set_render_shape(ctx, 1, r.opts, psi.BF16, 1, shape)
        out[shape] = r.backward(scene, gC, gF, gT)
        torch.cuda.synchronize()
        assert ctx.status_fetch()[0] == 0
    psi.psi_ctx_set_render_shape(ctx, 1, r.opts, psi.BF16, 1, 0)
    for shape in (8, 12):
        for k, ref in out[0].items():
            a, b = out[shape][k].double(), ref.double()
            assert torch.count_nonzero(b).item() > 0, k
            assert torch.linalg.norm(a - b).item() <= 1e-5 * torch.linalg.norm(b).item(), (shape, k)
