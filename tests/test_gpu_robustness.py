"""Non-finite inputs (needs a GPU): surfels whose centre, tangent axes, scales
or opacity hold NaN or infinity are culled in the projection (every cull test
is written so that a NaN fails it), so the frame equals, bit for bit, the
frame without them, and their gradients stay zero."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import multi_cams, opts_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _poison(w, seed=3):
    """Copies of the surfels with a seeded subset made non-finite, and that subset."""
    s = w.surfels
    rng = np.random.default_rng(seed)
    bad = np.sort(rng.choice(s.n, 40, replace=False))
    p = sg.Surfels(*(np.array(getattr(s, f)) for f in ("mu", "tu", "tv", "scale", "opacity", "rgb")))
    kinds = [("mu", 0, np.nan), ("mu", 2, np.inf), ("mu", 1, -np.inf), ("tu", 1, np.nan), ("tv", 0, np.nan),
             ("scale", 0, np.nan), ("scale", 1, np.inf), ("opacity", None, np.nan)]
    for j, i in enumerate(bad):
        f, c, v = kinds[j % len(kinds)]
        arr = getattr(p, f)
        if c is None:
            arr[i] = v
        else:
            arr[i, c] = v
    return p, bad


@pytest.mark.parametrize("K", [0, 8])
def test_nonfinite_surfels_are_culled(ctx, K):
    from paper_2604_10982_gb300 import pipeline as pl
    w = sg.dense_box(n=4000, d=16)
    poisoned, bad = _poison(w)
    keep = np.setdiff1d(np.arange(w.surfels.n), bad)
    clean = w.surfels.subset(keep)
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=K > 0)
    outs = []
    for s, f in ((poisoned, w.features), (clean, w.features[keep])):
        scene = pl.DeviceScene(s, f)
        r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=16)
        r.frame(scene)
        P = r.n_pix
        g = torch.Generator(device="cpu").manual_seed(2)
        gC, gF, gT = (torch.randn(3, P, generator=g).cuda(), torch.randn(P, 16, generator=g).cuda(),
                      torch.randn(P, generator=g).cuda())
        grads = r.backward(scene, gC, gF, gT)
        torch.cuda.synchronize()
        assert ctx.status_fetch()[0] == 0
        counts = r.counts[: len(cams) * s.n].view(len(cams), s.n).cpu().numpy()
        outs.append((r.rgb.cpu(), r.T.cpu(), r.F.cpu(), {k: v.cpu() for k, v in grads.items()}, counts))
    (rgb_p, T_p, F_p, g_p, c_p), (rgb_c, T_c, F_c, g_c, _) = outs
    assert (c_p[:, bad] == 0).all()
    assert torch.equal(rgb_p, rgb_c) and torch.equal(T_p, T_c) and torch.equal(F_p, F_c)
    for k in g_p:
        assert torch.count_nonzero(g_p[k][bad]).item() == 0, k
        a, b = g_p[k][keep].double(), g_c[k].double()
        assert torch.linalg.norm(a - b).item() <= 1e-5 * max(torch.linalg.norm(b).item(), 1e-30), k
