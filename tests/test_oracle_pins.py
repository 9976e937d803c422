"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from . import pins


@pytest.fixture(scope="module")
def box():
    return sg.dense_box(n=3000)


def test_fronto_parallel_closed_form(oracle_lib):
    pins.pin_fronto_parallel()


def test_rotated_surfel_point_recovered(oracle_lib):
    pins.pin_rotated_point()


def test_two_surfels_hand_computed(oracle_lib):
    pins.pin_two_surfels()


def test_early_termination_count(oracle_lib):
    pins.pin_termination()


def test_partition_of_unity(oracle_lib, box):
    pins.pin_partition_of_unity(box)


def test_topk_special_cases(oracle_lib, box):
    pins.pin_topk_special_cases(box)


def test_tile_coverage_bruteforce(oracle_lib, box):
    pins.pin_coverage(box)


def test_tile_coverage_opacity_radius(oracle_lib, box):
    pins.pin_coverage(box, modes=(orc.EXACT,), opacity_radius=True)


def test_conic_bounds_vs_sampled_boundary(oracle_lib, box):
    pins.pin_conic_bounds(box)


def test_ranges_vs_bincount(oracle_lib):
    pins.pin_ranges()


def test_rho_upper_bound(oracle_lib):
    pins.pin_rho()


def test_fd_gradients(oracle_lib):
    w = sg.crop_scene(n=500, d=32, size=64)
    checked, worst = pins.fd_check(w, params_per_kind=10)
    assert checked >= 40


def test_lowpass_filter_max_of_terms(oracle_lib):
    pins.pin_lowpass()


def test_tile_coverage_lowpass(oracle_lib):
    pins.pin_coverage(sg.dense_box(n=1500, scale_median=0.05), lowpass=True)


def test_fd_gradients_lowpass(oracle_lib):
    w = sg.crop_scene(n=500, d=16, size=64, scale_median=0.08)
    checked, worst = pins.fd_check(w, params_per_kind=8, lowpass=True)
    assert checked >= 32


def test_near_plane_cull_bruteforce(oracle_lib):
    crossing, beyond = pins.pin_near_plane()
    assert crossing >= 20 and beyond >= 20


def test_sphere_radius_semi_major(oracle_lib):
    n, rotated = pins.pin_sphere_radius()
    assert n >= 100 and rotated >= 20


def test_tiny_config_shape(oracle_lib):
    w = sg.tiny()
    assert w.surfels.n == 2000 and w.cameras[0].width == 128 and w.features.shape == (2000, 16)
    out = orc.render(w.surfels, w.cameras[0], orc.Opts(top_k=8), feat=w.features)
    assert np.max(np.abs(out["sumw"] + out["T"] - 1.0)) < 1e-12


@pytest.mark.parametrize("plant,check", [
    (1, "fronto"), (2, "two"), (3, "topk"), (4, "fd"), (5, "coverage"), (6, "lowpass"), (7, "fd_lowpass"),
    (8, "near"), (9, "sphere"), (10, "near"),
])
def test_planted_mistake_is_caught(plant, check):
    """A deliberately wrong oracle build fails the pin aimed at that mistake."""
    fn = {
        "fronto": pins.pin_fronto_parallel,
        "two": pins.pin_two_surfels,
        "topk": lambda: pins.pin_topk_special_cases(sg.dense_box(n=3000)),
        "fd": lambda: pins.fd_check(sg.crop_scene(n=200, d=8, size=48), params_per_kind=6),
        "coverage": lambda: pins.pin_coverage(sg.dense_box(n=3000), modes=(orc.EXACT,)),
        "lowpass": pins.pin_lowpass,
        "fd_lowpass": lambda: pins.fd_check(sg.crop_scene(n=300, d=8, size=48, scale_median=0.08),
                                            params_per_kind=6, lowpass=True),
        "near": pins.pin_near_plane,
        "sphere": pins.pin_sphere_radius,
    }[check]
    orc.use_variant(plant)
    try:
        with pytest.raises(AssertionError):
            fn()
    finally:
        orc.use_variant(0)


# ---------------------------------------------------------------- instance labels (Sec. 4.1, Eqs. 4-8)
def _label_case(seed=5, n=40, q=7, d=16):
    f = sg.make_features(n, d, seed).astype(np.float64)
    qf = sg.make_queries(q, d, seed).astype(np.float64) * 3.0
    mu, cov = sg.make_query_gaussians(q, seed, (-2, -2, 0), (2, 2, 3))
    p = np.stack([sg.uniform(seed, 20 + k, n) * 4 - 2 for k in range(3)], axis=1)
    return f, qf, mu.astype(np.float64), cov.astype(np.float64), p


def _labels_pinned(plant=0):
    """The label oracle against library routines that are not the oracle's:
    scipy's multivariate normal density (the geometric factor is a ratio of
    two of its values), its logistic function and its softmax."""
    from scipy.special import expit, softmax
    from scipy.stats import multivariate_normal
    f, qf, mu, cov, p = _label_case()
    L = orc.surfel_labels(f, qf, mu, cov, p, plant=plant)
    S = expit(f @ qf.T)
    D = np.stack([multivariate_normal(mu[k], cov[k]).pdf(p) / multivariate_normal(mu[k], cov[k]).pdf(mu[k])
                  for k in range(len(mu))], axis=1)
    ref = softmax(S * D, axis=1)
    return np.abs(L - ref).max()


def test_labels_against_library_densities():
    assert _labels_pinned() < 1e-12


def test_labels_special_cases():
    f, qf, mu, cov, p = _label_case()
    L = orc.surfel_labels(f, qf, mu, cov, p)
    # a distribution over the queries for every surfel
    assert np.all(L > 0) and np.allclose(L.sum(1), 1.0, atol=1e-14)
    # a surfel at a query's centre: geometric factor exactly 1 for that query
    p0 = np.repeat(mu[:1], 3, axis=0)
    L0 = orc.surfel_labels(f[:3], qf[:1], mu[:1], cov[:1], p0)
    assert np.array_equal(L0, np.ones((3, 1)))
    # identical queries: the uniform distribution
    Lu = orc.surfel_labels(f, np.repeat(qf[:1], 5, 0), np.repeat(mu[:1], 5, 0), np.repeat(cov[:1], 5, 0), p)
    assert np.allclose(Lu, 0.2, atol=1e-15)


def test_label_ids_rendered_mixture():
    # Eq. 8 blends label vectors; the identity is the argmax (lowest on ties)
    I = np.array([[0.1, 0.5, 0.4], [0.3, 0.3, 0.2], [0.0, 0.0, 0.0]])
    ids, gap = orc.label_ids(I, np.array([0.5, 0.2, 1.0]))
    assert list(ids) == [1, 0, -1] and np.isclose(gap[0], 0.1)


@pytest.mark.parametrize("plant", [1, 2, 3, 4])
def test_label_planted_mistake_is_caught(plant):
    # dropped 1/2, softmax over surfels, covariance for precision, no sigmoid
    assert _labels_pinned(plant) > 1e-6


# ---------------------------------------------------------------- regularisers (Sec. 4.2)
def _reg_case(n=60, seed=3):
    s = sg.dense_box(n=n).surfels
    rng = np.random.default_rng(seed)
    M = 9
    node_mu = rng.normal(size=(M, 3))
    nn = rng.normal(size=(M, 3))
    node_n = nn / np.linalg.norm(nn, axis=1, keepdims=True)
    node_of = rng.integers(-1, M, n)
    return s, node_of, node_mu, node_n


def _reg_loss(s, node_of, node_mu, node_n, lam, mu, tu, tv, sc, plant=0):
    t = sg.Surfels(mu=mu, tu=tu, tv=tv, scale=sc, opacity=s.opacity, rgb=s.rgb)
    Lg, Li, _ = orc.surfel_regularisers(t, node_of, node_mu, node_n, lam, plant=plant)
    return Lg + Li


def _reg_fd_error(plant=0, lam=0.7):
    """Hand-written gradients against central differences of the losses."""
    s, node_of, node_mu, node_n = _reg_case()
    base = dict(mu=np.asarray(s.mu, np.float64), tu=np.asarray(s.tu, np.float64), tv=np.asarray(s.tv, np.float64),
                sc=np.asarray(s.scale, np.float64))
    _, _, g = orc.surfel_regularisers(s, node_of, node_mu, node_n, lam, plant=plant)
    gmap = {"mu": g["mu"], "tu": g["tu"], "tv": g["tv"], "sc": g["scale"]}
    worst = 0.0
    h = 1e-6
    for key in ("mu", "tu", "tv", "sc"):
        for i in range(0, 60, 7):
            for c in range(base[key].shape[1]):
                p = {k2: v.copy() for k2, v in base.items()}
                m = {k2: v.copy() for k2, v in base.items()}
                p[key][i, c] += h
                m[key][i, c] -= h
                fd = (_reg_loss(s, node_of, node_mu, node_n, lam, p["mu"], p["tu"], p["tv"], p["sc"], plant) -
                      _reg_loss(s, node_of, node_mu, node_n, lam, m["mu"], m["tu"], m["tv"], m["sc"], plant)) / (2 * h)
                worst = max(worst, abs(fd - gmap[key][i, c]) / max(1.0, abs(fd)))
    return worst


def test_regulariser_gradients_against_central_differences():
    assert _reg_fd_error() < 1e-6


def test_regulariser_closed_forms():
    s, node_of, node_mu, node_n = _reg_case()
    # a surfel lying in its prior plane, facing along the prior normal, with equal scales: zero loss
    n0 = node_n[0]
    a = np.cross(n0, [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(n0, a)  # a x b = n0
    t = sg.Surfels(mu=(node_mu[0] + 0.3 * a)[None], tu=a[None], tv=b[None], scale=np.array([[0.1, 0.1]]),
                   opacity=np.array([0.5]), rgb=np.zeros((1, 3)))
    Lg, Li, _ = orc.surfel_regularisers(t, np.array([0]), node_mu, node_n, 0.7)
    assert abs(Lg) < 1e-15 and Li == 0.0
    # moved 0.25 along the normal and flipped (|n . nhat| = 1 still): distance term only
    t2 = sg.Surfels(mu=(node_mu[0] + 0.25 * n0)[None], tu=b[None], tv=a[None], scale=np.array([[0.3, 0.1]]),
                    opacity=np.array([0.5]), rgb=np.zeros((1, 3)))
    Lg2, Li2, _ = orc.surfel_regularisers(t2, np.array([0]), node_mu, node_n, 0.7)
    assert abs(Lg2 - 0.25) < 1e-14 and abs(Li2 - 0.04) < 1e-15
    # unassigned surfels carry no geometric loss
    Lg3, _, g3 = orc.surfel_regularisers(t2, np.array([-1]), node_mu, node_n, 0.7)
    assert Lg3 == 0.0 and not g3["mu"].any() and not g3["tu"].any()


@pytest.mark.parametrize("plant", [1, 2, 3])
def test_regulariser_planted_mistake_is_caught(plant):
    # no tangent projection of the normal gradient; signed alignment; |.| for the anisotropy square
    assert _reg_fd_error(plant) > 1e-4 or plant == 2 and _reg_plant2_closed_form_fails()


def _reg_plant2_closed_form_fails():
    s, node_of, node_mu, node_n = _reg_case()
    n0 = node_n[0]
    a = np.cross(n0, [1.0, 0.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(n0, a)
    t = sg.Surfels(mu=node_mu[0][None], tu=b[None], tv=a[None], scale=np.array([[0.1, 0.1]]),
                   opacity=np.array([0.5]), rgb=np.zeros((1, 3)))  # normal -nhat: |n . nhat| = 1
    Lg, _, _ = orc.surfel_regularisers(t, np.array([0]), node_mu, node_n, 0.7, plant=2)
    return abs(Lg) > 1e-6


# ---------------------------------------------------------------- quaternion frames
def _quats(n=50, seed=4):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, size=(n, 1))


def _frames_vs_scipy(plant=0):
    from scipy.spatial.transform import Rotation
    q = _quats()
    tu, tv = orc.quat_frames(q, plant=plant)
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy: scalar last, normalises
    return max(np.abs(tu - R[:, :, 0]).max(), np.abs(tv - R[:, :, 1]).max())


def test_quat_frames_against_scipy_rotation():
    assert _frames_vs_scipy() < 1e-14


def test_quat_frames_identity_and_orthonormal():
    tu, tv = orc.quat_frames(np.array([[3.0, 0.0, 0.0, 0.0]]))
    assert np.array_equal(tu, [[1.0, 0.0, 0.0]]) and np.array_equal(tv, [[0.0, 1.0, 0.0]])
    tu, tv = orc.quat_frames(_quats())
    assert np.allclose(np.sum(tu * tv, 1), 0.0, atol=1e-14) and np.allclose(np.linalg.norm(tu, axis=1), 1.0)


def test_quat_frames_gradient_central_differences():
    q = _quats()
    rng = np.random.default_rng(9)
    gu, gv = rng.normal(size=(50, 3)), rng.normal(size=(50, 3))
    g = orc.quat_frames_grad(q, gu, gv)
    h = 1e-6
    for k in range(4):
        p, m = q.copy(), q.copy()
        p[:, k] += h
        m[:, k] -= h
        fp = np.sum(orc.quat_frames(p)[0] * gu, 1) + np.sum(orc.quat_frames(p)[1] * gv, 1)
        fm = np.sum(orc.quat_frames(m)[0] * gu, 1) + np.sum(orc.quat_frames(m)[1] * gv, 1)
        assert np.abs((fp - fm) / (2 * h) - g[:, k]).max() < 1e-7


def test_quat_frames_planted_mistake_is_caught():
    assert _frames_vs_scipy(plant=1) > 1e-3


# ---------------------------------------------------------------- frustum cross-attention (Sec. 4.1)
def _attn_case(n=300, C=16, d=8, nq=5, seed=6):
    w = sg.dense_box(n=n, d=C)
    rng = np.random.default_rng(seed)
    W = [rng.normal(size=(C, d)) / np.sqrt(C) for _ in range(3)]
    Q = rng.normal(size=(nq, C))
    return w, w.features.astype(np.float64), Q, W


def test_attention_closed_forms():
    w, f, Q, (WQ, WK, WV) = _attn_case()
    cam = w.cameras[0]
    out, act, _ = orc.frustum_attention(w.surfels, f, cam, 0.2, Q, WQ, WK, WV)
    assert act.sum() > 10 and (~act).sum() > 0
    # W_K = 0: every score equal, the update is the mean value of the active set
    out0, _, _ = orc.frustum_attention(w.surfels, f, cam, 0.2, Q, WQ, np.zeros_like(WK), WV)
    assert np.allclose(out0, np.repeat((f[act] @ WV).mean(0, keepdims=True), len(Q), 0), atol=1e-12)
    # one active surfel: every query takes its value
    one = sg.Surfels(*(np.asarray(getattr(w.surfels, k))[act][:1] for k in ("mu", "tu", "tv", "scale", "opacity", "rgb")))
    o1, a1, _ = orc.frustum_attention(one, f[act][:1], cam, 0.2, Q, WQ, WK, WV)
    assert a1.all() and np.allclose(o1, np.repeat(f[act][:1] @ WV, len(Q), 0), atol=1e-12)


def test_attention_pos_enc_values():
    P = orc.attn_pos_enc(np.zeros((1, 3)), 12)
    # t = c // 3: even -> sin(0) = 0, odd -> cos(0) = 1
    assert np.array_equal(P[0], [0, 0, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1])
    x = np.array([[0.7, -1.2, 2.5]])
    P = orc.attn_pos_enc(x, 12)
    assert np.isclose(P[0, 0], np.sin(0.7)) and np.isclose(P[0, 4], np.cos(-1.2))
    w2 = np.exp(-np.log(10000.0) * 6.0 / 12.0)  # k = 1 from channel 6 on
    assert np.isclose(P[0, 8], np.sin(2.5 * w2)) and np.isclose(P[0, 10], np.cos(-1.2 * w2))


def test_frustum_test_is_conservative_by_sampling():
    """Brute force: sample each sphere; a surfel with any sample in front of
    the near plane projecting inside the image must be active."""
    w = sg.dense_box(n=400)
    cam = w.cameras[0]
    act, _ = orc.frustum_active(w.surfels, cam, 0.2)
    rng = np.random.default_rng(0)
    dirs = rng.normal(size=(400, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = np.sqrt(orc.CHI2_99_2D) * np.asarray(w.surfels.scale, np.float64).max(1)
    mu = np.asarray(w.surfels.mu, np.float64)
    R, t = np.asarray(cam.R, np.float64), np.asarray(cam.t, np.float64)
    for i in range(len(mu)):
        pts = mu[i] + rad[i] * dirs * rng.uniform(0, 1, size=(400, 1))
        x = pts @ R.T + t
        ok = x[:, 2] > 0.2
        u = cam.fx * x[ok, 0] / x[ok, 2] + cam.cx
        v = cam.fy * x[ok, 1] / x[ok, 2] + cam.cy
        inside = (u >= 0) & (u <= cam.width) & (v >= 0) & (v <= cam.height)
        if inside.any():
            assert act[i], i


def _two_surfel_closed_form(plant=0):
    """Two active surfels whose scores differ by exactly sqrt(d) ln 3: the
    softmax weights are 3/4 and 1/4, so Q' = 3/4 v_1 + 1/4 v_2 (W = I)."""
    w = sg.dense_box(n=400, d=4)
    cam = w.cameras[0]
    act, _ = orc.frustum_active(w.surfels, cam, 0.2)
    idx = np.nonzero(act)[0][:2]
    two = sg.Surfels(*(np.asarray(getattr(w.surfels, k))[idx] for k in ("mu", "tu", "tv", "scale", "opacity", "rgb")))
    C = d = 4
    I = np.eye(C)
    q = np.array([[1.0, 0.0, 0.0, 0.0]])
    K_want = np.array([[np.sqrt(d) * np.log(3.0), 0.3, -0.2, 0.5], [0.0, 0.1, 0.4, -0.6]])
    f = K_want - orc.attn_pos_enc(two.mu, C)  # so that K = f + psi(mu) = K_want
    out, a2, _ = orc.frustum_attention(two, f, cam, 0.2, q, I, I, I, plant=plant)
    assert a2.all()
    return np.abs(out - (0.75 * f[0] + 0.25 * f[1])[None]).max()


def test_attention_two_surfel_closed_form():
    assert _two_surfel_closed_form() < 1e-12


@pytest.mark.parametrize("plant", [1, 2])
def test_attention_planted_mistake_is_caught(plant):
    # missing 1/sqrt(d); softmax over queries instead of surfels
    assert _two_surfel_closed_form(plant) > 1e-3


def test_attention_gradients_central_differences():
    w, f, Q, (WQ, WK, WV) = _attn_case(n=120, C=12, d=6, nq=4)
    cam = w.cameras[0]
    rng = np.random.default_rng(2)
    G = rng.normal(size=(4, 6))
    g = orc.frustum_attention_grad(w.surfels, f, cam, 0.2, Q, WQ, WK, WV, G)
    act, margin = orc.frustum_active(w.surfels, cam, 0.2)
    mu0 = np.asarray(w.surfels.mu, np.float64)

    def L(Q_=Q, WQ_=WQ, WK_=WK, WV_=WV, f_=f, mu_=mu0):
        s = sg.Surfels(mu=mu_, tu=w.surfels.tu, tv=w.surfels.tv, scale=w.surfels.scale, opacity=w.surfels.opacity,
                       rgb=w.surfels.rgb)
        return float(np.sum(orc.frustum_attention(s, f_, cam, 0.2, Q_, WQ_, WK_, WV_)[0] * G))

    h = 1e-6
    for key, base in (("Q", Q), ("WQ", WQ), ("WK", WK), ("WV", WV), ("feat", f), ("mu", mu0)):
        for idx in [(0, 0), (1, 2), (base.shape[0] - 1, base.shape[1] - 1), (base.shape[0] // 2, 1)]:
            if key in ("feat", "mu") and (not act[idx[0]] or abs(margin[idx[0]]) < 1e-3):
                continue  # inactive surfels carry no gradient; avoid moving one across a plane
            p, m = base.copy(), base.copy()
            p[idx] += h
            m[idx] -= h
            arg = {"Q": "Q_", "WQ": "WQ_", "WK": "WK_", "WV": "WV_", "feat": "f_", "mu": "mu_"}[key]
            fd = (L(**{arg: p}) - L(**{arg: m})) / (2 * h)
            assert abs(fd - g[key][idx]) < 1e-6 * max(1.0, abs(fd)), (key, idx, fd, g[key][idx])


# ---------------------------------------------------------------- depth / normal table (2D-surfel geometry)
def _geometry_closed_forms(plant=0):
    """Camera-facing surfels: depth z0 and normal (0, 0, -1) whichever way the
    tangents are ordered; a tilted surfel: the normal from an independent
    rotation of the plane's spanning vectors."""
    from .pins import CAM, fronto_surfel
    a, _ = fronto_surfel(CAM, 0.1, -0.2, 2.5, 0.3, 0.2, 0.8)
    b = sg.Surfels(a.mu.copy(), a.tv.copy(), a.tu.copy(), a.scale.copy(), a.opacity.copy(), a.rgb.copy())
    err = 0.0
    for s in (a, b):
        G = orc.surfel_geometry(s, CAM, plant=plant)
        err = max(err, abs(G[0, 0] - 2.5), np.abs(G[0, 1:] - [0.0, 0.0, -1.0]).max())
    return err


def test_geometry_table_closed_forms_and_invariants():
    assert _geometry_closed_forms() < 1e-6
    w = sg.dense_box(n=500)
    cam = w.cameras[0]
    G = orc.surfel_geometry(w.surfels, cam)
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    xc = w.surfels.mu.astype(np.float64) @ R.T + np.asarray(cam.t, np.float64)
    assert np.allclose(G[:, 0], xc[:, 2], atol=0, rtol=0)
    assert np.allclose(np.linalg.norm(G[:, 1:], axis=1), 1.0, atol=1e-12)
    assert (np.sum(G[:, 1:] * xc, axis=1) <= 0).all()
    # normal is perpendicular to both camera-space tangents
    for f in ("tu", "tv"):
        tc = getattr(w.surfels, f).astype(np.float64) @ R.T
        assert np.abs(np.sum(tc * G[:, 1:], axis=1)).max() < 1e-6


def _geometry_fd_error(plant=0):
    w = sg.dense_box(n=40)
    cam = w.cameras[0]
    s64 = sg.Surfels(*(getattr(w.surfels, f).astype(np.float64) for f in ("mu", "tu", "tv", "scale", "opacity", "rgb")))
    g = sg.make_upstream(4 * s64.n, 9, 0).reshape(s64.n, 4).astype(np.float64)
    an = orc.surfel_geometry_grad(s64, cam, g, plant=plant)
    loss = lambda: float(np.sum(g * orc.surfel_geometry(s64, cam)))
    worst = 0.0
    for kind in ("mu", "tu", "tv"):
        arr = getattr(s64, kind)
        for i in range(0, s64.n, 7):
            for c in range(3):
                x0 = arr[i, c]
                h = 1e-6
                arr[i, c] = x0 + h; lp = loss()
                arr[i, c] = x0 - h; lm = loss()
                arr[i, c] = x0
                fd = (lp - lm) / (2 * h)
                worst = max(worst, abs(fd - an[kind][i, c]) / max(1.0, abs(fd)))
    return worst


def test_geometry_gradient_central_differences():
    assert _geometry_fd_error() < 1e-6


def test_geometry_planted_mistakes_are_caught():
    assert _geometry_closed_forms(plant=1) > 0.5        # no turn toward the camera
    assert _geometry_fd_error(plant=2) > 1e-3           # normalisation's projection dropped


def test_attention_empty_active_set_is_zero():
    """Reading: with no surfel in the frustum nothing is attended, Q' = 0, and
    every gradient vanishes."""
    w = sg.dense_box(n=300, d=16)
    cam = sg.look_camera((0.0, -6.0, 1.5), np.pi, 64, 64, 55.0)
    rng = np.random.default_rng(0)
    W = [rng.normal(size=(16, 4)) for _ in range(3)]
    Q, G = rng.normal(size=(3, 16)), rng.normal(size=(3, 4))
    out, act, _ = orc.frustum_attention(w.surfels, w.features, cam, 0.2, Q, *W)
    assert act.sum() == 0 and out.shape == (3, 4) and np.all(out == 0)
    g = orc.frustum_attention_grad(w.surfels, w.features, cam, 0.2, Q, *W, G)
    assert all(np.all(v == 0) for v in g.values())
