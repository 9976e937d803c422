"""psi_quantize_features against torch's own dtype conversions (needs a GPU):
BF16 and FP8-E4M3 (per-channel scale amax / 448, saturated) bit for bit,
including round-to-nearest-even ties, values near the saturation bound,
sub-normal results and an all-zero channel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _table(n, d, seed):
    rng = np.random.default_rng(seed)
    f = rng.normal(size=(n, d)).astype(np.float32) * np.exp(rng.uniform(-6, 3, d)).astype(np.float32)
    f[0, :] = 448.0                      # scale exactly 1 in every channel with |f| <= 448 ...
    f[1:, 1] = np.float32(2.0) ** -9 * np.arange(1, n) % 3   # sub-normal E4M3 results
    f[:, 2] = 0.0                        # an all-zero channel (scale from the 1e-30 floor)
    f[0, 2] = 0.0
    ties = np.array([1.0625, 1.1875, -2.125, 2.375, 416.0, 440.0, 447.9], np.float32)
    f[2:2 + len(ties), 3] = ties         # midpoints between E4M3 neighbours (scale 1)
    f[10, 4] = 448.0 * 1.0001            # scale above 1: f / scale rounds to 448
    # BF16 ties: exact midpoints between BF16 neighbours
    f[20:24, 5] = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -126 * (1 + 2 ** -8)], np.float32)
    return f


@pytest.mark.parametrize("n,d", [(1, 16), (4097, 64), (20_000, 128), (3001, 48), (777, 256)])
def test_quantize_matches_torch(ctx, n, d):
    from paper_2604_10982_gb300 import psi
    f = _table(max(n, 30), d, n + d)[:n].copy() if n >= 30 else _table(30, d, 1)[:n].copy()
    ft = torch.from_numpy(f)
    fd = ft.cuda()
    qb = torch.empty(n, d, dtype=torch.bfloat16, device="cuda")
    psi.psi_quantize_features(ctx, fd, n, d, psi.BF16, qb)
    q8 = torch.empty(n, d, dtype=torch.float8_e4m3fn, device="cuda")
    sc = torch.empty(d, dtype=torch.float32, device="cuda")
    psi.psi_quantize_features(ctx, fd, n, d, psi.FP8_E4M3, q8, sc)
    torch.cuda.synchronize()
    ref_b = ft.to(torch.bfloat16)
    assert torch.equal(qb.cpu().view(torch.int16), ref_b.view(torch.int16))
    amax = ft.abs().amax(0).clamp_min(1e-30)
    ref_s = (amax / 448.0).float()
    ref_q = (ft / ref_s).clamp(-448.0, 448.0).to(torch.float8_e4m3fn)
    assert torch.equal(sc.cpu().view(torch.int32), ref_s.view(torch.int32))
    assert torch.equal(q8.cpu().view(torch.uint8), ref_q.view(torch.uint8))


def test_quantize_rejects_bad_arguments(ctx):
    from paper_2604_10982_gb300 import psi
    f = torch.zeros(8, 24, device="cuda")
    q = torch.empty(8, 24, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(psi.PsiError):
        psi.psi_quantize_features(ctx, f, 8, 24, psi.BF16, q)
    f = torch.zeros(8, 32, device="cuda")
    q = torch.empty(8, 32, dtype=torch.float8_e4m3fn, device="cuda")
    with pytest.raises(psi.PsiError):
        psi.psi_quantize_features(ctx, f, 8, 32, psi.FP8_E4M3, q, None)
