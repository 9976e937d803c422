"""Launch-shape autotuner of the compositing kernels (needs a GPU): every shape
gives the same forward bit for bit and the same adjoint up to the order of
float32 atomic additions; the tuner stores its choice in the context."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import multi_cams, opts_of

pytestmark = pytest.mark.gpu

KEYS = ("mu", "tu", "tv", "scale", "opacity", "rgb", "feat")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


@pytest.fixture(scope="module")
def box():
    return sg.dense_box(n=6000, d=32)


def _setup(ctx, w, K, lowpass=False):
    from paper_2604_10982_gb300 import pipeline as pl
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=K > 0, lowpass=lowpass)
    scene = pl.DeviceScene(w.surfels, w.features)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=32, want_topk_ids=K > 0)
    r.frame(scene)
    P = r.n_pix
    g = torch.Generator(device="cpu").manual_seed(4)
    up = (torch.randn(3, P, generator=g).cuda(), torch.randn(P, 32, generator=g).cuda(), torch.randn(P, generator=g).cuda())
    return scene, r, up


def _outputs(r):
    outs = [r.rgb.clone(), r.T.clone(), r.n_last.clone(), r.F.clone()]
    if r.topk_ids is not None:
        outs += [r.topk_ids.clone(), r.topk_w.clone()]
    return outs


def _valid(K, D=32, pair_walk=False):
    return [s for s in range(16) if (not (s & 2) or (K == 0 and D % 32 == 0)) and (not (s & 8) or pair_walk)]


@pytest.mark.parametrize("K,lowpass", [(0, False), (8, False), (16, False), (8, True)])
def test_every_shape_same_result(ctx, box, K, lowpass):
    from paper_2604_10982_gb300 import psi
    scene, r, (gC, gF, gT) = _setup(ctx, box, K, lowpass)
    ref_f, ref_g = None, None
    for shape in _valid(K, pair_walk=K > 0):
        for which, saved in ((0, 0), (1, 1), (1, 0)):
            psi.psi_ctx_set_render_shape(ctx, which, r.opts, psi.F32, saved, shape)
            assert psi.psi_ctx_get_render_shape(ctx, which, r.opts, psi.F32, saved) == shape
        r.render(scene)
        outs = _outputs(r)
        g_saved = r.backward(scene, gC, gF, gT)
        g_re = r.backward(scene, gC, gF, gT, recompute=True)
        torch.cuda.synchronize()
        assert ctx.status_fetch()[0] == 0
        if ref_f is None:
            ref_f, ref_g = outs, g_saved
        for a, b in zip(outs, ref_f):
            assert torch.equal(a, b), shape
        for gg in (g_saved, g_re):
            for k in KEYS:
                a, b = gg[k].double(), ref_g[k].double()
                assert torch.linalg.norm(a - b).item() <= 1e-5 * max(torch.linalg.norm(b).item(), 1e-30), (shape, k)
    for which, saved in ((0, 0), (1, 1), (1, 0)):
        psi.psi_ctx_set_render_shape(ctx, which, r.opts, psi.F32, saved, 0)


@pytest.mark.parametrize("K", [0, 8])
def test_tuner_stores_fastest_and_zeroes_grads(ctx, box, K):
    from paper_2604_10982_gb300 import psi
    scene, r, (gC, gF, gT) = _setup(ctx, box, K)
    n = scene.n
    shapes = dict(mu=(n, 3), tu=(n, 3), tv=(n, 3), scale=(n, 2), opacity=(n,), rgb=(n, 3), feat=(n, 32))
    grads = {k: torch.full(shapes[k], 7.0, device="cuda") for k in KEYS}
    rep = r.tune(scene, gC, gF, gT, grads=grads, reps=2)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    for which, key, saved in ((0, "fwd", 0), (1, "bwd", 1)):
        ms, best = rep[key]
        valid = _valid(K, pair_walk=which == 1 and K > 0)
        assert best in valid
        assert all(ms[s] > 0 for s in valid) and all(ms[s] == -1 for s in range(16) if s not in valid)
        assert ms[best] == min(ms[s] for s in valid)
        assert psi.psi_ctx_get_render_shape(ctx, which, r.opts, psi.F32, saved) == best
    for k in KEYS:
        assert torch.count_nonzero(grads[k]).item() == 0, k
    # the outputs hold a valid frame: the same as a plain render with the tuned shape
    outs = _outputs(r)
    r.render(scene)
    torch.cuda.synchronize()
    for a, b in zip(outs, _outputs(r)):
        assert torch.equal(a, b)
    for which, saved in ((0, 0), (1, 1)):
        psi.psi_ctx_set_render_shape(ctx, which, r.opts, psi.F32, saved, 0)


def test_tuner_refuses_stream_capture(ctx, box):
    from paper_2604_10982_gb300 import psi
    scene, r, (gC, gF, gT) = _setup(ctx, box, 8)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            try:
                r.tune(scene, gC, gF, gT, reps=1, stream=s)
            except psi.PsiError as e:
                err = e
    assert err is not None and err.code == psi.PSI_ERR_INVALID_ARG
