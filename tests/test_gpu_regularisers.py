"""Geometric and anisotropy regularisers (Sec. 4.2) against the oracle (needs a GPU)."""
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


@pytest.mark.parametrize("n", [1, 1000, 100_003])
def test_regularisers_match_oracle(ctx, n):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    s = sg.dense_box(n=n).surfels
    rng = np.random.default_rng(n)
    M = 37
    node_mu = rng.normal(size=(M, 3)).astype(np.float32)
    nn = rng.normal(size=(M, 3))
    node_n = (nn / np.linalg.norm(nn, axis=1, keepdims=True)).astype(np.float32)
    node_of = rng.integers(-1, M, n).astype(np.int32)
    lam, wg, wi = 0.7, 1.3, 0.4
    scene = pl.DeviceScene(s, None)
    grads = {k: torch.zeros(n, d, device="cuda") for k, d in (("mu", 3), ("tu", 3), ("tv", 3), ("scale", 2))}
    gs = psi.PsiGrads(psi._ptr(grads["mu"]), psi._ptr(grads["tu"]), psi._ptr(grads["tv"]), psi._ptr(grads["scale"]),
                      None, None, None)
    losses = torch.empty(2, dtype=torch.float64, device="cuda")
    dev = lambda a: torch.from_numpy(a).cuda()
    psi.psi_surfel_regularisers(ctx, scene.surfels_struct(), dev(node_of), dev(node_mu), dev(node_n), M, lam, wg, wi,
                                losses, gs)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    Lg, Li, g = orc.surfel_regularisers(s, node_of, node_mu.astype(np.float64), node_n.astype(np.float64), lam)
    L = losses.cpu().numpy()
    assert abs(L[0] - Lg) <= 1e-5 * max(1.0, abs(Lg)) and abs(L[1] - Li) <= 1e-5 * max(1.0, abs(Li))
    for key, w in (("mu", wg), ("tu", wg), ("tv", wg), ("scale", wi)):
        ref = w * g[key]
        got = grads[key].cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max()), key


def test_regularisers_bad_node_index(ctx):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    s = sg.dense_box(n=10).surfels
    scene = pl.DeviceScene(s, None)
    node_of = torch.full((10,), 5, dtype=torch.int32, device="cuda")  # only 2 nodes
    mu = torch.zeros(2, 3, device="cuda")
    nrm = torch.tensor([[0.0, 0.0, 1.0]] * 2, device="cuda")
    losses = torch.empty(2, dtype=torch.float64, device="cuda")
    gs = psi.PsiGrads(None, None, None, None, None, None, None)
    psi.psi_surfel_regularisers(ctx, scene.surfels_struct(), node_of, mu, nrm, 2, 0.5, 1.0, 1.0, losses, gs)
    st, _ = ctx.status_fetch()
    assert st == psi.PSI_ERR_INVALID_ARG
