"""CUDA path vs the oracle, element by element (needs a GPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import GROSS, flags, multi_cams, opts_of

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


def _renderer(ctx, w, cams, o, D=0, F_dtype=0, feat_dtype=0, topk_ids=False):
    from paper_2604_10982_gb300 import pipeline as pl
    scene = pl.DeviceScene(w.surfels, w.features if D else None, feat_dtype=feat_dtype)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=D, F_dtype=F_dtype, want_topk_ids=topk_ids)
    return scene, r


@pytest.mark.parametrize("mode", [orc.SPHERE, orc.AABB, orc.EXACT])
@pytest.mark.parametrize("oprad", [False, True])
def test_project_counts_and_bounds_bitexact(ctx, box, mode, oprad):
    cams = multi_cams()
    o = orc.Opts(mode=mode, opacity_radius=oprad)
    scene, r = _renderer(ctx, box, cams, o)
    r.project(scene)
    torch.cuda.synchronize()
    n = box.surfels.n
    counts = r.counts.cpu().numpy().view(np.uint32)
    bins = r.bins.cpu().numpy()[: len(cams) * n * 32].view(np.uint32).reshape(len(cams) * n, 8)
    for v, cam in enumerate(cams):
        b = orc.bin_view(box.surfels, cam, o)
        c = counts[v * n:(v + 1) * n]
        assert np.array_equal(c, b["count"]), (v, int((c != b["count"]).sum()))
        vis = b["count"] > 0
        g = bins[v * n:(v + 1) * n][vis]
        ell = b["ell"][vis].view(np.uint32)
        for k, name in enumerate(["ex", "ey", "A00", "A01", "A11"]):
            assert np.array_equal(g[:, k], ell[:, k]), name
        assert np.array_equal(g[:, 5], b["depth_bits"][vis])
        rect = b["rect"][vis].astype(np.uint32)
        assert np.array_equal(g[:, 6], rect[:, 0] | (rect[:, 1] << 16))
        assert np.array_equal(g[:, 7], rect[:, 2] | (rect[:, 3] << 16))


@pytest.mark.parametrize("mode", [orc.SPHERE, orc.AABB, orc.EXACT])
def test_project_near_plane_straddles_bitexact(ctx, mode):
    """Surfels whose support disc crosses the near plane while the centre is
    beyond it (the pinned near-plane cull), at random tilts: counts, ellipse
    and rectangle bit for bit, emitted keys in emission order."""
    w = sg.near_plane(seed=21, n=600)
    cam = w.cameras[0]
    o = orc.Opts(mode=mode)
    scene, r = _renderer(ctx, w, [cam], o)
    r.project(scene)
    r.intersect()
    torch.cuda.synchronize()
    n = w.surfels.n
    b = orc.bin_view(w.surfels, cam, o)
    counts = r.counts.cpu().numpy().view(np.uint32)[:n]
    assert np.array_equal(counts, b["count"]), int((counts != b["count"]).sum())
    assert 0 < int((b["count"] > 0).sum()) < n
    bins = r.bins.cpu().numpy()[: n * 32].view(np.uint32).reshape(n, 8)
    vis = b["count"] > 0
    ell = b["ell"][vis].view(np.uint32)
    assert np.array_equal(bins[vis][:, :5], ell[:, :5])
    P = int(r.num_pairs.item())
    ek, ev = orc.emit_pairs(w.surfels, [cam], o)
    assert P == len(ek)
    assert np.array_equal(r.keys[:P].cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(r.vals[:P].cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("mode", [orc.SPHERE, orc.AABB, orc.EXACT])
def test_keys_sort_ranges_bitexact(ctx, box, mode):
    cams = multi_cams()
    o = orc.Opts(mode=mode, opacity_radius=(mode == orc.EXACT))
    scene, r = _renderer(ctx, box, cams, o)
    r.project(scene)
    r.intersect()
    torch.cuda.synchronize()
    P = int(r.num_pairs.item())
    ek, ev = orc.emit_pairs(box.surfels, cams, o)
    assert P == len(ek)
    gk = r.keys[:P].cpu().numpy().view(np.uint64)
    gv = r.vals[:P].cpu().numpy().view(np.uint32)
    assert np.array_equal(gk, ek) and np.array_equal(gv, ev), "emission order differs"
    r.sort()
    torch.cuda.synchronize()
    sk, sv = orc.sort_pairs(ek, ev)
    gk = r.keys[:P].cpu().numpy().view(np.uint64)
    gv = r.vals[:P].cpu().numpy().view(np.uint32)
    assert np.array_equal(gk, sk) and np.array_equal(gv, sv), "sorted order differs"
    rall = r.ranges.cpu().numpy().view(np.uint32)
    rg = rall[: 2 * r.n_tiles].reshape(-1, 2).astype(np.int64)
    ro = orc.tile_ranges(sk, r.n_tiles).astype(np.int64)
    # launch order: a permutation of the tiles, longest lists first (by octave)
    order = rall[2 * r.n_tiles: 3 * r.n_tiles].astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(r.n_tiles))
    ln = (ro[:, 1] - ro[:, 0])[order]
    assert (np.diff(np.floor(np.log2(np.maximum(ln, 1)))) <= 0).all()
    assert np.array_equal(rg[:, 1] - rg[:, 0], ro[:, 1] - ro[:, 0])
    nonempty = ro[:, 1] > ro[:, 0]
    assert np.array_equal(rg[nonempty], ro[nonempty])
    st, _ = ctx.status_fetch()
    assert st == 0


def test_sort_random_keys_vs_stable_argsort(ctx):
    """The radix sort alone on random keys with many duplicates, odd sizes."""
    from paper_2604_10982_gb300 import psi
    rng = np.random.default_rng(5)
    for n, bits in [(1, 40), (4095, 45), (4097, 33), (100_003, 45), (257_000, 49)]:
        hi = rng.integers(0, 1 << (bits - 32), n, dtype=np.uint64)
        lo = rng.integers(0, 64, n, dtype=np.uint64)  # heavy duplication
        keys = (hi << np.uint64(32)) | lo
        vals = np.arange(n, dtype=np.uint32)
        dk = torch.from_numpy(keys.view(np.int64)).cuda()
        dv = torch.from_numpy(vals.view(np.int32)).cuda()
        cap = n + 100
        kk = torch.zeros(cap, dtype=torch.int64, device="cuda"); kk[:n] = dk
        vv = torch.zeros(cap, dtype=torch.int32, device="cuda"); vv[:n] = dv
        npairs = torch.tensor([n], dtype=torch.int64, device="cuda")
        ws = torch.empty(psi.sort_workspace_size(cap), dtype=torch.uint8, device="cuda")
        nt = 1 << (bits - 32)
        ranges = torch.empty(nt * 3, dtype=torch.int32, device="cuda")
        psi.psi_sort_keys(ctx, kk, vv, npairs, cap, 0, bits, ranges, nt, ws)
        torch.cuda.synchronize()
        perm = np.argsort(keys, kind="stable")
        assert np.array_equal(kk[:n].cpu().numpy().view(np.uint64), keys[perm])
        assert np.array_equal(vv[:n].cpu().numpy().view(np.uint32), vals[perm])


def test_sort_count_beyond_capacity_is_clamped(ctx):
    """*d_num_pairs larger than the buffers: the first `capacity` pairs are
    sorted and ranged, PSI_ERR_CAPACITY is raised with the requested count,
    and nothing past capacity is touched."""
    from paper_2604_10982_gb300 import psi
    rng = np.random.default_rng(9)
    cap, bits = 70_001, 40
    keys = (rng.integers(0, 1 << (bits - 32), cap, dtype=np.uint64) << np.uint64(32)) | \
        rng.integers(0, 1 << 20, cap, dtype=np.uint64)
    vals = np.arange(cap, dtype=np.uint32)
    guard = 4096
    kk = torch.full((cap + guard,), -7, dtype=torch.int64, device="cuda")
    vv = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    kk[:cap] = torch.from_numpy(keys.view(np.int64)).cuda()
    vv[:cap] = torch.from_numpy(vals.view(np.int32)).cuda()
    npairs = torch.tensor([cap + 5], dtype=torch.int64, device="cuda")
    ws = torch.empty(psi.sort_workspace_size(cap), dtype=torch.uint8, device="cuda")
    nt = 1 << (bits - 32)
    ranges = torch.empty(nt * 3, dtype=torch.int32, device="cuda")
    ctx.status_fetch()
    psi.psi_sort_keys(ctx, kk, vv, npairs, cap, 0, bits, ranges, nt, ws)
    st, detail = ctx.status_fetch()
    assert st == psi.PSI_ERR_CAPACITY and detail == cap + 5, (st, detail)
    perm = np.argsort(keys, kind="stable")
    assert np.array_equal(kk[:cap].cpu().numpy().view(np.uint64), keys[perm])
    assert np.array_equal(vv[:cap].cpu().numpy().view(np.uint32), vals[perm])
    assert (kk[cap:] == -7).all() and (vv[cap:] == -7).all()
    rg = ranges[: 2 * nt].cpu().numpy().view(np.uint32).reshape(nt, 2).astype(np.int64)
    cnt = np.bincount((keys >> np.uint64(32)).astype(np.int64), minlength=nt)
    assert np.array_equal(rg[:, 1] - rg[:, 0], cnt)


def _compare_render(r, scene, w, cams, o, D, feat64, bf16_out=False):
    rgb = r.rgb.cpu().numpy().astype(np.float64)
    T = r.T.cpu().numpy().astype(np.float64)
    F = r.F.float().cpu().numpy().astype(np.float64) if (D and r.F is not None) else None
    ids = r.topk_ids.cpu().numpy() if r.topk_ids is not None else None
    stats = {}
    for v, cam in enumerate(cams):
        a, b = int(r.pix_base[v]), int(r.pix_base[v + 1])
        ref = orc.render(w.surfels, cam, o, feat=feat64)
        straddle, illcond, neartie = flags(ref, cam)
        ok = ~(straddle | illcond)
        assert ok.mean() > 0.98, (v, ok.mean())
        e_rgb = np.abs(rgb[:, a:b].T - ref["rgb"]).max(1)
        e_T = np.abs(T[a:b] - ref["T"])
        assert e_rgb[ok].max() < 1e-4, (v, e_rgb[ok].max())
        assert e_T[ok].max() < 1e-4, (v, e_T[ok].max())
        # gross errors are not excused anywhere
        assert e_rgb.max() < GROSS and e_T.max() < GROSS, (v, e_rgb.max(), e_T.max())
        if ids is not None:
            g = ids[a:b]
            same = np.array([set(g[p][g[p] >= 0]) == set(ref["topk"][p][ref["topk"][p] >= 0]) for p in range(b - a)])
            bad = ok & ~neartie & ~same
            assert bad.sum() == 0, (v, int(bad.sum()))
        if F is not None:
            okF = ok & ~neartie
            tol = 1e-4 if not bf16_out else None
            e_F = np.abs(F[a:b] - ref["F"]).max(1)
            if bf16_out:
                rel = e_F / (np.abs(ref["F"]).max(1) + 1e-3)
                assert rel[okF].max() < 2e-2, (v, rel[okF].max())
            else:
                assert e_F[okF].max() < tol, (v, e_F[okF].max())
                assert e_F[~neartie].max() < 10 * GROSS, (v, e_F.max())
        stats[v] = dict(excused=float(1 - ok.mean()), neartie=int(neartie.sum()), max_rgb=float(e_rgb.max()))
    return stats


@pytest.mark.parametrize("mode", [orc.SPHERE, orc.AABB, orc.EXACT])
def test_render_dense_f32(ctx, box, mode):
    cams = multi_cams()
    o = orc.Opts(mode=mode, top_k=0)
    scene, r = _renderer(ctx, box, cams, o, D=32)
    r.frame(scene)
    torch.cuda.synchronize()
    _compare_render(r, scene, box, cams, o, 32, box.features.astype(np.float64))


@pytest.mark.parametrize("K", [1, 4, 8, 16, 32])
def test_render_topk_f32(ctx, box, K):
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=True)
    scene, r = _renderer(ctx, box, cams, o, D=32, topk_ids=True)
    r.frame(scene)
    torch.cuda.synchronize()
    _compare_render(r, scene, box, cams, o, 32, box.features.astype(np.float64))


def test_topk_large_k_equals_dense_bitwise(ctx, box):
    """K >= #contributors: Top-K features equal the dense ones bit for bit."""
    cams = multi_cams()[:1]
    o_d = orc.Opts(mode=orc.EXACT, top_k=0)
    o_k = orc.Opts(mode=orc.EXACT, top_k=32)
    ref = orc.render(box.surfels, cams[0], orc.Opts(top_k=0))
    scene, rd = _renderer(ctx, box, cams, o_d, D=32)
    rd.frame(scene)
    _, rk = _renderer(ctx, box, cams, o_k, D=32)
    rk.frame(scene)
    torch.cuda.synchronize()
    nl = rd.n_last.cpu().numpy()
    cnt = ref["ncontrib"]
    sel = cnt <= 32
    assert torch.equal(rd.rgb, rk.rgb) and torch.equal(rd.T, rk.T)
    Fd, Fk = rd.F.cpu().numpy(), rk.F.cpu().numpy()
    assert np.array_equal(Fd[sel], Fk[sel])
    assert (nl >= 0).all()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_render_quantised_features(ctx, box, dtype):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    cams = multi_cams()[:2]
    fdt = psi.BF16 if dtype == "bf16" else psi.FP8_E4M3
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene, r = _renderer(ctx, box, cams, o, D=32, feat_dtype=fdt)
    r.frame(scene)
    torch.cuda.synchronize()
    deq = pl.dequantize(scene.q, scene.qscale, fdt)
    # against the oracle fed the same stored values: FP32 accumulation only
    _compare_render(r, scene, box, cams, o, 32, deq)
    # against the unquantised FP32 oracle: the storage error (reported)
    ref = orc.render(box.surfels, cams[0], o, feat=box.features.astype(np.float64))
    F = r.F.float().cpu().numpy()[: cams[0].width * cams[0].height]
    m = ref["sumw"] > 0.5
    rel = np.linalg.norm(F[m] - ref["F"][m]) / np.linalg.norm(ref["F"][m])
    assert rel < (2e-2 if dtype == "bf16" else 8e-2), rel


def test_render_bf16_output(ctx, box):
    from paper_2604_10982_gb300 import psi
    cams = multi_cams()[:1]
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene, r = _renderer(ctx, box, cams, o, D=32, F_dtype=psi.BF16, feat_dtype=psi.BF16)
    r.frame(scene)
    torch.cuda.synchronize()
    from paper_2604_10982_gb300 import pipeline as pl
    _compare_render(r, scene, box, cams, o, 32, pl.dequantize(scene.q, None, psi.BF16), bf16_out=True)


def test_tiny_config_parity(ctx):
    w = sg.tiny()
    o = orc.Opts(mode=orc.EXACT, top_k=8)
    scene, r = _renderer(ctx, w, w.cameras, o, D=16, topk_ids=True)
    r.frame(scene)
    torch.cuda.synchronize()
    _compare_render(r, scene, w, w.cameras, o, 16, w.features.astype(np.float64))


def test_empty_and_degenerate_inputs(ctx):
    """No surfels; all culled (behind the camera); a single huge surfel."""
    from paper_2604_10982_gb300 import pipeline as pl
    cam = sg.look_camera((0.0, -6.0, 1.5), 0.0, 40, 24, 40.0)
    o = orc.Opts(mode=orc.EXACT, top_k=4)
    for n in (0, 1):
        w = sg.dense_box(n=max(n, 1), d=16)
        s = w.surfels if n else w.surfels.subset(np.arange(0))
        feats = w.features[:n]
        ws = sg.Workload("t", s, [cam], 16, 4, feats)
        scene = pl.DeviceScene(s, feats if n else None)
        r = pl.Renderer(ctx, s.n, [cam], opts_of(o), capacity=4096, D=16 if n else 0)
        r.frame(scene)
        torch.cuda.synchronize()
        ref = orc.render(s, cam, o, feat=feats.astype(np.float64) if n else None)
        assert np.abs(r.rgb.cpu().numpy().T - ref["rgb"]).max() < 1e-4
        assert np.abs(r.T.cpu().numpy() - ref["T"]).max() < 1e-4
    # behind the camera: everything culled, image empty
    w = sg.dense_box(n=500, d=16)
    back = sg.look_camera((0.0, -6.0, 1.5), np.pi, 40, 24, 40.0)
    scene = pl.DeviceScene(w.surfels, w.features)
    r = pl.Renderer(ctx, w.surfels.n, [back], opts_of(o), capacity=4096, D=16)
    r.frame(scene)
    torch.cuda.synchronize()
    assert int(r.num_pairs.item()) == 0
    assert float(r.rgb.abs().max()) == 0.0 and float((r.T - 1).abs().max()) == 0.0


def test_capacity_overflow_reported(ctx, box):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    cams = multi_cams()[:1]
    scene = pl.DeviceScene(box.surfels, None)
    r = pl.Renderer(ctx, box.surfels.n, cams, opts_of(orc.Opts()), capacity=100)
    r.project(scene)
    r.intersect()
    st, req = ctx.status_fetch()
    assert st == psi.PSI_ERR_CAPACITY and req > 100
    assert int(r.num_pairs.item()) == 100
    st, _ = ctx.status_fetch()
    assert st == 0


def _long_list_scene():
    """Large, dense surfels seen by a small view: tile lists of thousands of
    entries (many 256-record batches) and early termination of every pixel."""
    w = sg.dense_box(n=20000, d=16, width=64, height=48, scale_median=0.25)
    return w


def test_render_long_lists_early_exit(ctx):
    w = _long_list_scene()
    o = orc.Opts(mode=orc.AABB, top_k=8)
    scene, r = _renderer(ctx, w, w.cameras, o, D=16, topk_ids=True)
    r.frame(scene)
    torch.cuda.synchronize()
    st, site = ctx.status_fetch()
    assert st == 0, (st, site)
    rg = r.ranges.cpu().numpy().view(np.uint32)[: 2 * r.n_tiles].reshape(-1, 2).astype(np.int64)
    assert (rg[:, 1] - rg[:, 0]).max() > 3 * 256  # several batches per tile
    _compare_render(r, scene, w, w.cameras, o, 16, w.features.astype(np.float64))
