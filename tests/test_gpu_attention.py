"""Frustum-constrained cross-attention (Sec. 4.1) against the oracle (needs a GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _run(ctx, w, cam, dtype, nq, d, seed=1):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    C = w.features.shape[1]
    rng = np.random.default_rng(seed)
    W = [(rng.normal(size=(C, d)) / np.sqrt(C)).astype(np.float32) for _ in range(3)]
    Q = rng.normal(size=(nq, C)).astype(np.float32)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=dtype)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty(nq, d, device="cuda")
    ws = torch.empty(psi.attention_workspace_size(scene.n, C, d, nq), dtype=torch.uint8, device="cuda")
    camarr = psi.cameras([cam])
    psi.psi_frustum_attention(ctx, scene.surfels_struct(), scene.features_struct(), camarr[0], 0.2, dev(Q), nq,
                              dev(W[0]), dev(W[1]), dev(W[2]), d, out, ws)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    feat = pl.dequantize(scene.q, scene.qscale, dtype) if dtype != psi.F32 else w.features.astype(np.float64)
    ref, act, margin = orc.frustum_attention(w.surfels, feat, cam, 0.2, Q.astype(np.float64), *W)
    return out.cpu().numpy().astype(np.float64), ref, act, margin


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_attention_matches_oracle(ctx, dtype):
    from paper_2604_10982_gb300 import psi
    w = sg.dense_box(n=5000, d=64)
    cam = w.cameras[0]
    got, ref, act, margin = _run(ctx, w, cam, psi.F32 if dtype == "f32" else psi.BF16, 7, 32)
    # the float32 frustum test agrees with the FP64 one away from the planes
    assert np.min(np.abs(margin)) > 1e-4, "a surfel sits on a frustum plane: pick another seed"
    assert 0 < act.sum() < len(act)
    assert np.abs(got - ref).max() <= 2e-4 * max(1.0, np.abs(ref).max())


def test_attention_street_view(ctx):
    """200k surfels of the street, one 720p view: most surfels outside the
    frustum. Surfels within 1e-4 m of a frustum plane (where float32 and FP64
    may decide differently) are left out of the input, by the oracle's margin."""
    import dataclasses
    from paper_2604_10982_gb300 import psi
    w = sg.street()
    cam = w.cameras[0]
    _, margin = orc.frustum_active(w.surfels, cam, 0.2)
    keep = np.abs(margin) >= 1e-4
    s = sg.Surfels(*(np.ascontiguousarray(np.asarray(getattr(w.surfels, k))[keep])
                     for k in ("mu", "tu", "tv", "scale", "opacity", "rgb")))
    w2 = dataclasses.replace(w, surfels=s, features=np.ascontiguousarray(w.features[keep]))
    got, ref, act, _ = _run(ctx, w2, cam, psi.F32, 100, 64)
    assert act.mean() < 0.9 and keep.mean() > 0.999
    assert np.abs(got - ref).max() <= 5e-4 * max(1.0, np.abs(ref).max())


def test_attention_gradients_match_oracle(ctx):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=4000, d=32)
    cam = w.cameras[0]
    C, d, nq = 32, 16, 6
    rng = np.random.default_rng(3)
    W = [(rng.normal(size=(C, d)) / np.sqrt(C)).astype(np.float32) for _ in range(3)]
    Q = rng.normal(size=(nq, C)).astype(np.float32)
    G = rng.normal(size=(nq, d)).astype(np.float32)
    scene = pl.DeviceScene(w.surfels, w.features)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty(nq, d, device="cuda")
    ws = torch.empty(psi.attention_workspace_size(scene.n, C, d, nq), dtype=torch.uint8, device="cuda")
    Qd, Wd = dev(Q), [dev(x) for x in W]
    psi.psi_frustum_attention(ctx, scene.surfels_struct(), scene.features_struct(), psi.cameras([cam])[0], 0.2, Qd,
                              nq, *Wd, d, out, ws)
    gQ, gWQ, gWK, gWV = torch.empty(nq, C, device="cuda"), *(torch.empty(C, d, device="cuda") for _ in range(3))
    gfeat = torch.zeros(scene.n, C, device="cuda")
    gmu = torch.zeros(scene.n, 3, device="cuda")
    gs = psi.PsiGrads(psi._ptr(gmu), None, None, None, None, None, psi._ptr(gfeat))
    psi.psi_frustum_attention_bwd(ctx, scene.surfels_struct(), scene.features_struct(), Qd, nq, *Wd, d, dev(G),
                                  gQ, gWQ, gWK, gWV, gs, ws)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    _, margin = orc.frustum_active(w.surfels, cam, 0.2)
    assert np.min(np.abs(margin)) > 1e-4
    ref = orc.frustum_attention_grad(w.surfels, w.features.astype(np.float64), cam, 0.2, Q, *W, G)
    for key, got in (("Q", gQ), ("WQ", gWQ), ("WK", gWK), ("WV", gWV), ("feat", gfeat), ("mu", gmu)):
        g = got.cpu().numpy().astype(np.float64)
        r = ref[key]
        assert np.linalg.norm(g - r) <= 1e-4 * max(np.linalg.norm(r), 1e-12), key
