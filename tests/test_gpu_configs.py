"""The full-size workloads against the oracle (needs a GPU): bit-exact keys
and sorted order over whole frames, values on sampled pixels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import check_values, opts_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def _sampled_parity(r, w, cams, o, feat64, n_per_view=64, seed=0, bf16_rel=None, max_excused=0.25):
    """Sampled pixels of every view against the oracle (see check_values).
    At 1080p many surfels are sub-pixel at grazing angles, so a larger share of
    pixels is ill-conditioned than in the small scenes; those are held to the
    FP32 error model instead of 1e-4."""
    rgb = r.rgb.cpu().numpy().astype(np.float64)
    T = r.T.cpu().numpy().astype(np.float64)
    F = r.F.float().cpu().numpy().astype(np.float64) if (r.F is not None and feat64 is not None) else None
    rng = np.random.default_rng(seed)
    shares = []
    for v, cam in enumerate(cams):
        a = int(r.pix_base[v])
        P = cam.width * cam.height
        idx = rng.choice(P, min(n_per_view, P), replace=False)
        ref = orc.render(w.surfels, cam, o, feat=feat64, pixels=orc.all_pixels(cam)[idx])
        shares.append(check_values(rgb[:, a + idx].T, T[a + idx], None if F is None else F[a + idx], ref, cam,
                                   bf16_rel=bf16_rel, max_excused=1.0,
                                   fmax=0.0 if feat64 is None else np.abs(feat64).max()))
    assert np.mean(shares) <= max_excused, shares
    return shares


def test_street_720p_modes_keys_bitexact(ctx):
    """200k surfels, 1280x720, D=64 FP32, K=16: SPHERE / AABB / EXACT lists
    bit-exact over the whole frame; fewer keys per tile at each step."""
    from paper_2604_10982_gb300 import pipeline as pl
    w = sg.street()
    cam = w.cameras[0]
    scene = pl.DeviceScene(w.surfels, w.features)
    pairs = {}
    for mode in (orc.SPHERE, orc.AABB, orc.EXACT):
        o = orc.Opts(mode=mode, top_k=16)
        r = pl.make_renderer(ctx, scene, [cam], opts_of(o), D=64)
        r.frame(scene)
        torch.cuda.synchronize()
        P = int(r.num_pairs.item())
        ek, ev = orc.emit_pairs(w.surfels, [cam], o)
        sk, sv = orc.sort_pairs(ek, ev)
        assert P == len(sk)
        assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), sk)
        assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), sv)
        pairs[mode] = P
        if mode == orc.EXACT:
            _sampled_parity(r, w, [cam], o, w.features.astype(np.float64), n_per_view=256)
    assert pairs[orc.EXACT] < pairs[orc.AABB] < pairs[orc.SPHERE]


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_batch_16_views_one_launch_and_graph(ctx, dtype):
    """1M surfels, 16 views of uneven resolution in one launch per stage,
    D=128 in BF16 / FP8-E4M3 with per-channel scales; keys bit-exact over all
    views; values on sampled pixels of every view; a CUDA-graph replay gives
    identical outputs."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.batch_scene()
    cams = w.cameras
    fdt = psi.BF16 if dtype == "bf16" else psi.FP8_E4M3
    o = orc.Opts(mode=orc.EXACT, top_k=16, opacity_radius=True)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=fdt)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=128)
    r.frame(scene)
    torch.cuda.synchronize()
    st, _ = ctx.status_fetch()
    assert st == 0
    P = int(r.num_pairs.item())
    if dtype == "bf16":
        ek, ev = orc.emit_pairs(w.surfels, cams, o)
        sk, sv = orc.sort_pairs(ek, ev)
        assert P == len(sk)
        assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), sk)
        assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), sv)
    deq = pl.dequantize(scene.q, scene.qscale, fdt)
    _sampled_parity(r, w, cams, o, deq, n_per_view=24)
    # storage error against the unquantised features (reported bound)
    idx = np.random.default_rng(3).choice(cams[2].width * cams[2].height, 64, replace=False)
    ref = orc.render(w.surfels, cams[2], o, feat=w.features.astype(np.float64), pixels=orc.all_pixels(cams[2])[idx])
    F = r.F.float().cpu().numpy()[int(r.pix_base[2]) + idx]
    m = ref["sumw"] > 0.5
    rel = np.linalg.norm(F[m] - ref["F"][m]) / np.linalg.norm(ref["F"][m])
    assert rel < (2e-2 if dtype == "bf16" else 8e-2), rel
    # graph capture of the whole batched frame, replayed
    rgb0, F0 = r.rgb.clone(), r.F.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        r.frame(scene)
    r.rgb.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(r.rgb, rgb0) and torch.equal(r.F, F0)


def test_panoptic_full_size_sampled(ctx):
    """3M surfels, 1920x1080, D=128 BF16, K=8, Q=100: 2048 sampled pixels of
    the rendered frame against the oracle -- colour and T to 1e-4, the BF16
    feature map to 2e-2 relative, the Top-K id sets equal -- on every pixel
    that is not excused; the excused shares (threshold straddles,
    ill-conditioned pixels, near ties) are reported with the largest error over
    them, and held to their own bounds. Decoded ids on 4096 pixels against an
    FP64 matmul of the GPU's own feature map."""
    from paper_2604_10982_gb300 import pipeline as pl, psi
    from .gpu_common import GROSS, cond_bound, flags
    w = sg.panoptic_scene(frames=2)
    cam = w.cameras[0]
    o = orc.Opts(mode=orc.EXACT, top_k=8, opacity_radius=True)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16)
    r = pl.make_renderer(ctx, scene, [cam], opts_of(o), D=128, F_dtype=psi.BF16, want_topk_ids=True)
    r.frame(scene)
    Q = torch.from_numpy(w.queries).cuda().to(torch.bfloat16)
    ids = torch.empty(r.n_pix, dtype=torch.int32, device="cuda")
    psi.psi_decode_queries(ctx, r.F, r.n_pix, 128, Q, 100, r.T, ids)
    torch.cuda.synchronize()
    assert ctx.status_fetch()[0] == 0
    deq = pl.dequantize(scene.q, None, psi.BF16)
    idx = np.random.default_rng(11).choice(r.n_pix, 2048, replace=False)
    ref = orc.render(w.surfels, cam, o, feat=deq, pixels=orc.all_pixels(cam)[idx])
    rgb = r.rgb.cpu().numpy().astype(np.float64)[:, idx].T
    T = r.T.cpu().numpy().astype(np.float64)[idx]
    F = r.F.float().cpu().numpy().astype(np.float64)[idx]
    tk = r.topk_ids.cpu().numpy()[idx]
    st, ic, nt = flags(ref, cam)
    strict = ~(st | ic)
    e_px = np.maximum(np.abs(rgb - ref["rgb"]).max(1), np.abs(T - ref["T"]))
    relF = np.abs(F - ref["F"]).max(1) / (np.abs(ref["F"]).max(1) + 1e-3)
    same = np.array([set(tk[p][tk[p] >= 0].tolist()) == set(ref["topk"][p][ref["topk"][p] >= 0].tolist())
                     for p in range(len(idx))])
    icm = ic & ~st
    report = dict(pixels=len(idx), straddle=float(st.mean()), ill_conditioned=float(icm.mean()),
                  near_tie=float(nt.mean()), max_err_strict=float(e_px[strict].max(initial=0)),
                  max_err_ill_conditioned=float(e_px[icm].max(initial=0)),
                  max_err_straddle=float(e_px[st].max(initial=0)),
                  topk_set_mismatch_strict=int((strict & ~nt & ~same).sum()),
                  topk_set_mismatch_excused=int((~(strict & ~nt) & ~same).sum()),
                  max_relF_strict=float(relF[strict & ~nt].max(initial=0)))
    print("panoptic 1080p parity:", report)
    assert report["max_err_strict"] < 1e-4, report
    assert report["max_relF_strict"] < 2e-2, report
    assert report["topk_set_mismatch_strict"] == 0, report
    assert (e_px[icm] < cond_bound(ref, cam)[icm]).all(), report
    assert e_px.max() < GROSS, report
    assert (~strict).mean() <= 0.25, report
    # decode of the GPU's own feature map on sampled pixels (FP64 matmul)
    idx = np.random.default_rng(7).choice(r.n_pix, 4096, replace=False)
    Fs = r.F.float().cpu().numpy()[idx].astype(np.float64)
    rid, L, gap = orc.decode(Fs, Q.float().cpu().numpy().astype(np.float64), r.T.cpu().numpy()[idx])
    gid = ids.cpu().numpy()[idx]
    tie = gap < 1e-4 * (np.abs(L).max(1) + 1e-6)
    assert ((gid != rid) & ~tie).sum() == 0
