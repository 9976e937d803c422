"""Tensor-core query decode vs FP64 matmul + argmax (needs a GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import opts_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _check(F_bf16, Q_bf16, T, ids, logits, n_q):
    F64 = F_bf16.float().cpu().numpy().astype(np.float64)
    Q64 = Q_bf16.float().cpu().numpy().astype(np.float64)
    rid, L, gap = orc.decode(F64, Q64, T.cpu().numpy())
    gid = ids.cpu().numpy()
    scale = np.abs(L).max(1) + 1e-6
    tie = gap < 1e-4 * scale  # FP32 accumulation order may flip these
    bad = (gid != rid) & ~tie
    assert bad.sum() == 0, (int(bad.sum()), np.nonzero(bad)[0][:10])
    if logits is not None:
        gl = logits.float().cpu().numpy().astype(np.float64)
        # BF16 rounding of the FP32 accumulator: half an ulp of bf16 plus accumulation error
        err = np.abs(gl - L)
        assert (err <= np.abs(L) * 2.0 ** -8 + 1e-4 * scale[:, None]).all(), err.max()
    return int(tie.sum())


@pytest.mark.parametrize("D", [64, 128])
@pytest.mark.parametrize("n_q", [1, 16, 37, 100, 128])
def test_decode_random(ctx, D, n_q):
    from paper_2604_10982_gb300 import psi
    n_pix = 1000 + 77  # 8 full tiles of 128 and a ragged tail
    g = torch.Generator().manual_seed(D * 1000 + n_q)
    F = torch.randn(n_pix, D, generator=g).to(torch.bfloat16).cuda()
    Q = (torch.randn(n_q, D, generator=g) / D ** 0.5).to(torch.bfloat16).cuda()
    T = torch.rand(n_pix, generator=g).cuda()
    T[::7] = 1.0  # nothing rendered there
    ids = torch.full((n_pix,), -7, dtype=torch.int32, device="cuda")
    logits = torch.empty(n_pix, n_q, dtype=torch.bfloat16, device="cuda")  # odd n_q: unaligned rows
    psi.psi_decode_queries(ctx, F, n_pix, D, Q, n_q, T, ids, logits)
    torch.cuda.synchronize()
    assert (ids.cpu().numpy()[::7] == -1).all()
    _check(F, Q, T, ids, logits, n_q)
    st, _ = ctx.status_fetch()
    assert st == 0


def test_decode_large_many_ctas(ctx):
    from paper_2604_10982_gb300 import psi
    n_pix, D, n_q = 300_001, 128, 100
    g = torch.Generator().manual_seed(11)
    F = torch.randn(n_pix, D, generator=g).to(torch.bfloat16).cuda()
    Q = (torch.randn(n_q, D, generator=g) / D ** 0.5).to(torch.bfloat16).cuda()
    T = torch.zeros(n_pix).cuda()
    ids = torch.full((n_pix,), -7, dtype=torch.int32, device="cuda")
    psi.psi_decode_queries(ctx, F, n_pix, D, Q, n_q, T, ids, None)
    torch.cuda.synchronize()
    _check(F, Q, T, ids, None, n_q)


def test_decode_of_rendered_features(ctx):
    """Decode the GPU's own rendered BF16 feature map (isolates a6 from a4)."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=6000, d=128)
    cams = [w.cameras[0]]
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=128, F_dtype=psi.BF16)
    r.frame(scene)
    Qn = sg.make_queries(100, 128, 0)
    Q = torch.from_numpy(Qn).to(torch.bfloat16).cuda()
    ids = torch.empty(r.n_pix, dtype=torch.int32, device="cuda")
    logits = torch.empty(r.n_pix, 100, dtype=torch.bfloat16, device="cuda")
    psi.psi_decode_queries(ctx, r.F, r.n_pix, 128, Q, 100, r.T, ids, logits)
    torch.cuda.synchronize()
    _check(r.F, Q, r.T, ids, logits, 100)
    empty = (1 - r.T.cpu().numpy()) < 1e-4
    assert empty.any() and (~empty).any()


def test_decode_rejects_bad_args(ctx):
    from paper_2604_10982_gb300 import psi
    F = torch.zeros(10, 96, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(psi.PsiError):
        psi.psi_decode_queries(ctx, F, 10, 96, F, 4, torch.zeros(10, device="cuda"),
                               torch.zeros(10, dtype=torch.int32, device="cuda"))
