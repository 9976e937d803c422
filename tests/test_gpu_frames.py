"""Quaternion-parameterised tangent frames and their adjoint against the oracle (needs a GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


@pytest.mark.parametrize("n", [1, 257, 100_000])
def test_frames_and_adjoint(ctx, n):
    from paper_2604_10982_gb300 import psi
    rng = np.random.default_rng(n)
    q = (rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, size=(n, 1))).astype(np.float32)
    gu = rng.normal(size=(n, 3)).astype(np.float32)
    gv = rng.normal(size=(n, 3)).astype(np.float32)
    qd = torch.from_numpy(q).cuda()
    tu = torch.empty(n, 3, device="cuda")
    tv = torch.empty(n, 3, device="cuda")
    gq = torch.full((n, 4), 0.25, device="cuda")  # accumulated into
    psi.psi_quat_frames(ctx, qd, n, tu, tv)
    psi.psi_quat_frames_bwd(ctx, qd, n, torch.from_numpy(gu).cuda(), torch.from_numpy(gv).cuda(), gq)
    torch.cuda.synchronize()
    rtu, rtv = orc.quat_frames(q.astype(np.float64))
    assert np.abs(tu.cpu().numpy() - rtu).max() < 2e-6 and np.abs(tv.cpu().numpy() - rtv).max() < 2e-6
    rg = orc.quat_frames_grad(q.astype(np.float64), gu, gv) + 0.25
    scale = np.abs(rg).max(axis=1, keepdims=True)
    assert (np.abs(gq.cpu().numpy() - rg) / np.maximum(scale, 1.0)).max() < 5e-6
