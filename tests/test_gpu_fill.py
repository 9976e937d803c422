"""psi_grads_zero (needs a GPU): every float of every given gradient buffer
becomes 0, nothing outside them changes, whatever the buffers' alignment and
length (head before the first 16-byte boundary, 16-byte body, tail)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


WIDTHS = dict(mu=3, tu=3, tv=3, scale=2, opacity=1, rgb=3)


@pytest.mark.parametrize("n,dim,offset", [(1, 16, 0), (7, 16, 1), (1001, 32, 3), (65537, 128, 2), (300000, 48, 1)])
def test_zero_every_member_and_nothing_else(ctx, n, dim, offset):
    from paper_2604_10982_gb300 import psi
    widths = dict(WIDTHS, feat=dim)
    guard = 8
    bufs, views = {}, {}
    for i, (k, wdt) in enumerate(widths.items()):
        # one buffer per member with guard floats on both sides; the member
        # starts `offset + i` floats into it, so the alignments differ
        start = guard + offset + i
        b = torch.full((start + n * wdt + guard,), 5.0, device="cuda")
        bufs[k] = (b, start)
        views[k] = b[start:start + n * wdt]
    g = psi.PsiGrads(*(psi._ptr(views[k]) for k in ("mu", "tu", "tv", "scale", "opacity", "rgb", "feat")))
    psi.psi_grads_zero(ctx, g, n, dim)
    torch.cuda.synchronize()
    for k, (b, start) in bufs.items():
        assert torch.count_nonzero(views[k]).item() == 0, k
        assert torch.all(b[:start] == 5.0).item() and torch.all(b[start + n * widths[k]:] == 5.0).item(), k


def test_null_members_and_empty_sizes(ctx):
    from paper_2604_10982_gb300 import psi
    feat = torch.full((10, 16), 3.0, device="cuda")
    mu = torch.full((10, 3), 3.0, device="cuda")
    g = psi.PsiGrads(psi._ptr(mu), None, None, None, None, None, psi._ptr(feat))
    psi.psi_grads_zero(ctx, g, 0, 16)  # n = 0: nothing to do
    torch.cuda.synchronize()
    assert torch.all(mu == 3.0).item() and torch.all(feat == 3.0).item()
    psi.psi_grads_zero(ctx, g, 10, 0)  # dim = 0: the feature gradient is empty
    torch.cuda.synchronize()
    assert torch.count_nonzero(mu).item() == 0 and torch.all(feat == 3.0).item()
    with pytest.raises(psi.PsiError):
        psi.psi_grads_zero(ctx, g, -1, 16)
