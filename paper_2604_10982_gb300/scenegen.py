"""Seeded synthetic inputs: plane-structured surfel scenes, cameras and upstream
gradients.

This module only draws random numbers and places primitives on planes. It
holds none of the rendering arithmetic, and both the CUDA path and the CPU
oracle consume exactly the arrays it returns.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): output i of
stream s is ``mix64(key_s + (i + 1) * GAMMA)``, computed in uint64 with
wrap-around. Uniforms are the top 53 bits scaled by 2**-53; normals use the
Box-Muller transform in double precision. Everything is computed in double
and stored as float32, so a scene is a pure function of (seed, sizes).

The surfel model follows the paper's map representation (Sec. 3.1: 2D surfels
on planar structure, Sec. 3.2: plane-constrained initialisation). Scenes stand
in for the paper's datasets, which are not available: ground and facade planes,
centres uniform on a plane with N(0, 2 cm) jitter along its normal, normals
tilted by N(0, 5 deg) about a random in-plane axis, log-normal tangent scales
(median 5 cm, log-sigma 0.5), opacity sigmoid(N(0,1)), colour U[0,1]^3 and
features N(0,1)^D.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.array([(int(seed) & 0xFFFFFFFF) << 32 | (int(stream) & 0xFFFFFFFF)], dtype=np.uint64)
        return _mix64(base + _GAMMA)[0]


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from stream ``stream`` of ``seed`` (counter-based)."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = _mix64(key + ctr * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals: Box-Muller on uniform pairs (u1, u2) of the stream,
    normal 2k = r cos(2 pi u2), 2k+1 = r sin(2 pi u2), r = sqrt(-2 ln(1-u1))."""
    k0 = offset // 2
    k1 = (offset + n + 1) // 2
    u = uniform(seed, stream, 2 * (k1 - k0), 2 * k0)
    r = np.sqrt(-2.0 * np.log(1.0 - u[0::2]))
    th = 2.0 * math.pi * u[1::2]
    z = np.empty(2 * (k1 - k0))
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    s = offset - 2 * k0
    return z[s:s + n]


# stream ids (one per drawn quantity)
_S_PLANE, _S_A, _S_B, _S_OFF, _S_AXIS, _S_TILT, _S_PSI, _S_SU, _S_SV, _S_OP, _S_RGB, _S_FEAT, _S_QUERY = range(13)
_S_GRAD = 40
_S_CAMJIT = 60
_S_NEAR = 70  # streams 70..77: the near-plane scene


@dataclass
class Plane:
    origin: tuple
    e1: tuple
    e2: tuple
    l1: float
    l2: float

    @property
    def area(self) -> float:
        return self.l1 * self.l2


def box_planes():
    """Ground z=0 (x in [-4,4], y in [-5,5]) and facades x=+-4 (z in [0,10])."""
    return [
        Plane((-4.0, -5.0, 0.0), (1, 0, 0), (0, 1, 0), 8.0, 10.0),
        Plane((-4.0, -5.0, 0.0), (0, 1, 0), (0, 0, 1), 10.0, 10.0),
        Plane((4.0, -5.0, 0.0), (0, 1, 0), (0, 0, 1), 10.0, 10.0),
    ]


def street_planes():
    """Ground (x in [-8,8], y in [0,60]) and facades x=+-8 (z in [0,12])."""
    return [
        Plane((-8.0, 0.0, 0.0), (1, 0, 0), (0, 1, 0), 16.0, 60.0),
        Plane((-8.0, 0.0, 0.0), (0, 1, 0), (0, 0, 1), 60.0, 12.0),
        Plane((8.0, 0.0, 0.0), (0, 1, 0), (0, 0, 1), 60.0, 12.0),
    ]


@dataclass
class Surfels:
    """Structure-of-arrays surfel set, all float32, C-contiguous."""
    mu: np.ndarray      # [N,3] centre (world, metres)
    tu: np.ndarray      # [N,3] first tangent axis
    tv: np.ndarray      # [N,3] second tangent axis
    scale: np.ndarray   # [N,2] (s_u, s_v)
    opacity: np.ndarray  # [N]
    rgb: np.ndarray     # [N,3]

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    def subset(self, idx: np.ndarray) -> "Surfels":
        return Surfels(*(np.ascontiguousarray(a[idx]) for a in
                         (self.mu, self.tu, self.tv, self.scale, self.opacity, self.rgb)))


def make_surfels(n: int, planes, seed: int, scale_median: float = 0.05) -> Surfels:
    areas = np.array([p.area for p in planes], dtype=np.float64)
    cum = np.cumsum(areas) / areas.sum()
    pick = np.searchsorted(cum, uniform(seed, _S_PLANE, n), side="right")
    pick = np.minimum(pick, len(planes) - 1)
    org = np.array([p.origin for p in planes], dtype=np.float64)[pick]
    e1 = np.array([p.e1 for p in planes], dtype=np.float64)[pick]
    e2 = np.array([p.e2 for p in planes], dtype=np.float64)[pick]
    l1 = np.array([p.l1 for p in planes], dtype=np.float64)[pick]
    l2 = np.array([p.l2 for p in planes], dtype=np.float64)[pick]
    nrm = np.cross(e1, e2)
    a = uniform(seed, _S_A, n) * l1
    b = uniform(seed, _S_B, n) * l2
    mu = org + a[:, None] * e1 + b[:, None] * e2 + (0.02 * normal(seed, _S_OFF, n))[:, None] * nrm
    # tilt the normal by N(0, 5 deg) about a uniformly random in-plane axis
    phi = 2.0 * math.pi * uniform(seed, _S_AXIS, n)
    axis = np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2
    th = np.deg2rad(5.0) * normal(seed, _S_TILT, n)
    n2 = nrm * np.cos(th)[:, None] + np.cross(axis, nrm) * np.sin(th)[:, None]
    b1 = axis
    b2 = np.cross(n2, b1)
    psi = 2.0 * math.pi * uniform(seed, _S_PSI, n)
    tu = np.cos(psi)[:, None] * b1 + np.sin(psi)[:, None] * b2
    tv = np.cross(n2, tu)
    su = np.exp(math.log(scale_median) + 0.5 * normal(seed, _S_SU, n))
    sv = np.exp(math.log(scale_median) + 0.5 * normal(seed, _S_SV, n))
    op = 1.0 / (1.0 + np.exp(-normal(seed, _S_OP, n)))
    rgb = uniform(seed, _S_RGB, 3 * n).reshape(n, 3)
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    return Surfels(f32(mu), f32(tu), f32(tv), f32(np.stack([su, sv], 1)), f32(op), f32(rgb))


def make_features(n: int, d: int, seed: int, chunk: int = 1 << 22) -> np.ndarray:
    """[N, D] float32 features ~ N(0,1), generated in independent chunks of the
    counter-based stream (threads in parallel; numpy releases the GIL)."""
    import concurrent.futures as cf
    import os
    out = np.empty((n, d), dtype=np.float32)
    flat = out.reshape(-1)
    total = n * d

    def fill(s):
        m = min(chunk, total - s)
        flat[s:s + m] = normal(seed, _S_FEAT, m, offset=s)

    starts = list(range(0, total, chunk))
    if len(starts) <= 1:
        for s in starts:
            fill(s)
    else:
        with cf.ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 4, 32)) as ex:
            list(ex.map(fill, starts))
    return out


def make_queries(q: int, d: int, seed: int) -> np.ndarray:
    """[Q, D] float32 query vectors ~ N(0,1)/sqrt(D)."""
    return (normal(seed, _S_QUERY, q * d).reshape(q, d) / math.sqrt(d)).astype(np.float32)


def make_query_gaussians(q: int, seed: int, lo, hi, sigma_range=(0.5, 3.0)):
    """Spatial Gaussians of Q instance queries (Sec. 4.1): centres uniform in
    the box [lo, hi], covariances R diag(s^2) R^T with per-axis s uniform in
    sigma_range and R a rotation about a uniformly random axis by a uniform
    angle. Returns (mu [Q,3], cov [Q,3,3]) float32."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    u = uniform(seed, _S_QUERY + 1, q * 10).reshape(q, 10)
    mu = lo + u[:, 0:3] * (hi - lo)
    s = sigma_range[0] + u[:, 3:6] * (sigma_range[1] - sigma_range[0])
    cov = np.zeros((q, 3, 3))
    for k in range(q):
        z = 2.0 * u[k, 6] - 1.0
        ph = 2.0 * math.pi * u[k, 7]
        axis = np.array([math.sqrt(1 - z * z) * math.cos(ph), math.sqrt(1 - z * z) * math.sin(ph), z])
        ang = 2.0 * math.pi * u[k, 8]
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
        cov[k] = R @ np.diag(s[k] ** 2) @ R.T
    return mu.astype(np.float32), cov.astype(np.float32)


def make_upstream(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """n float32 N(0,1) values used as an upstream loss gradient."""
    return normal(seed, _S_GRAD + stream, n).astype(np.float32)


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward), x_c = R x_w + t.

    Pixel (px, py) samples the continuous image point (px + 1/2, py + 1/2)."""
    R: np.ndarray  # [3,3]
    t: np.ndarray  # [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        """float32 [18]: R (row-major 9), t (3), fx, fy, cx, cy, W, H."""
        return np.concatenate([np.asarray(self.R, np.float64).reshape(9), np.asarray(self.t, np.float64).reshape(3),
                               [self.fx, self.fy, self.cx, self.cy, self.width, self.height]]).astype(np.float32)


def look_camera(pos, yaw: float, width: int, height: int, f: float) -> Camera:
    """Camera at ``pos`` looking along (-sin yaw, cos yaw, 0) (yaw 0 looks down +y)."""
    fwd = np.array([-math.sin(yaw), math.cos(yaw), 0.0])
    right = np.array([math.cos(yaw), math.sin(yaw), 0.0])
    down = np.array([0.0, 0.0, -1.0])
    R = np.stack([right, down, fwd]).astype(np.float32).astype(np.float64)
    t = (-(R @ np.asarray(pos, np.float64))).astype(np.float32).astype(np.float64)
    return Camera(R, t, float(f), float(f), width / 2.0, height / 2.0, int(width), int(height))


# ----------------------------------------------------------------- workloads
@dataclass
class Workload:
    name: str
    surfels: Surfels
    cameras: list
    feat_dim: int
    top_k: int
    features: np.ndarray | None = None
    queries: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def tiny(seed: int = 0, n: int = 2000, d: int = 16) -> Workload:
    """2k surfels in a 10 m box, one 128x128 view (f=110), D=16, K=8."""
    s = make_surfels(n, box_planes(), seed)
    cam = look_camera((0.0, -6.0, 1.5), 0.0, 128, 128, 110.0)
    return Workload("tiny-2k-128x128-D16-K8", s, [cam], d, 8, make_features(n, d, seed))


def dense_box(seed: int = 1, n: int = 6000, d: int = 32, width: int = 150, height: int = 100,
              scale_median: float = 0.12, top_k: int = 8) -> Workload:
    """Parity scene: the box of ``tiny`` with larger, denser surfels, seen by a
    ragged 150x100 view (9.4 x 6.25 tiles of 16x16), so that many pixels have
    more than K contributors and the image spans several tiles and a ragged tail."""
    s = make_surfels(n, box_planes(), seed, scale_median=scale_median)
    cam = look_camera((0.0, -6.0, 1.5), 0.0, width, height, 0.86 * width)
    return Workload(f"densebox-{n}-{width}x{height}-D{d}-K{top_k}", s, [cam], d, top_k, make_features(n, d, seed))


def near_plane(seed: int = 11, n: int = 400, d: int = 16) -> Workload:
    """Surfels close to the box camera of ``tiny`` (128x128, f=110) at random
    tilts: centres in camera space at depth U[0.21, 0.9] m inside the central
    60 % of the image, normals uniform on the sphere, scales log-uniform in
    [5 mm, 25 cm], opacity 0.9. The near plane z=0.2 m cuts the support disc
    of many of them while their centres lie beyond it."""
    cam = look_camera((0.0, -6.0, 1.5), 0.0, 128, 128, 110.0)
    u = lambda k, m: uniform(seed, _S_NEAR + k, m)
    z = 0.21 + 0.69 * u(0, n)
    xc = np.stack([(0.6 * u(1, n) - 0.3) * z, (0.6 * u(2, n) - 0.3) * z, z], 1)
    nrm = normal(seed, _S_NEAR + 3, 3 * n).reshape(n, 3)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    a = np.cross(nrm, normal(seed, _S_NEAR + 4, 3 * n).reshape(n, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(nrm, a)
    sc = np.exp(math.log(0.005) + (math.log(0.25) - math.log(0.005)) * u(5, 2 * n)).reshape(n, 2)
    R, t = cam.R, cam.t
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    s = Surfels(f32((xc - t) @ R), f32(a @ R), f32(b @ R), f32(sc), f32(np.full(n, 0.9)), f32(u(6, 3 * n).reshape(n, 3)))
    return Workload(f"nearplane-{n}-128x128", s, [cam], d, 8, make_features(n, d, seed))


def street(seed: int = 0, n: int = 200_000, d: int = 64) -> Workload:
    """200k surfels on a 60 m street, one 1280x720 view (f=640), D=64, K=16."""
    s = make_surfels(n, street_planes(), seed)
    cam = look_camera((0.0, 2.0, 1.5), 0.0, 1280, 720, 640.0)
    return Workload("street-200k-1280x720-D64-K16", s, [cam], d, 16, make_features(n, d, seed))


def grad_scene(seed: int = 0, n: int = 500_000, d: int = 128) -> Workload:
    """500k surfels, one 960x540 view (f=480), D=128, K=16."""
    s = make_surfels(n, street_planes(), seed)
    cam = look_camera((0.0, 5.0, 1.5), 0.0, 960, 540, 480.0)
    return Workload("grad-500k-960x540-D128-K16", s, [cam], d, 16, make_features(n, d, seed))


def crop_scene(seed: int = 0, n: int = 500, d: int = 128, size: int = 64, scale_median: float = 0.05) -> Workload:
    """A 64x64 crop camera (f=480) with 500 street surfels inside its frustum."""
    cam = look_camera((0.0, 5.0, 1.5), 0.0, size, size, 480.0)
    pool = make_surfels(40 * n, street_planes(), seed, scale_median=scale_median)
    xc = pool.mu.astype(np.float64) @ cam.R.T + cam.t
    z = xc[:, 2]
    ok = z > 0.5
    px = np.where(ok, cam.fx * xc[:, 0] / np.where(ok, z, 1) + cam.cx, -1e9)
    py = np.where(ok, cam.fy * xc[:, 1] / np.where(ok, z, 1) + cam.cy, -1e9)
    inside = ok & (px > -4) & (px < size + 4) & (py > -4) & (py < size + 4)
    idx = np.nonzero(inside)[0][:n]
    s = pool.subset(idx)
    return Workload(f"crop-{s.n}-{size}x{size}-D{d}-K16", s, [cam], d, 16, make_features(s.n, d, seed))


_RES = [(640, 360), (960, 540), (1280, 720), (1600, 900), (1920, 1080)]


def batch_scene(seed: int = 0, n: int = 1_000_000, d: int = 128, views: int = 16) -> Workload:
    """1M surfels, 16 views of cycled resolution on a 60 m trajectory (hfov 90 deg)."""
    s = make_surfels(n, street_planes(), seed)
    jit = (uniform(seed, _S_CAMJIT, views) * 2.0 - 1.0) * math.radians(10.0)
    cams = []
    for i in range(views):
        w, h = _RES[i % len(_RES)]
        yaw = (0.0 if i % 2 == 0 else math.pi) + jit[i]
        cams.append(look_camera((0.0, 60.0 * i / max(views - 1, 1), 1.5), yaw, w, h, w / 2.0))
    return Workload(f"batch-{n // 1000}k-{views}views-D{d}", s, cams, d, 16, make_features(n, d, seed))


def panoptic_scene(seed: int = 0, n: int = 3_000_000, d: int = 128, frames: int = 32, q: int = 100,
                   with_features: bool = True) -> Workload:
    """3M surfels, 32 frames of 1920x1080 (f=960) from y=5 to y=55, D=128, K=8, Q=100."""
    s = make_surfels(n, street_planes(), seed)
    cams = [look_camera((0.0, 5.0 + 50.0 * i / max(frames - 1, 1), 1.5), 0.0, 1920, 1080, 960.0)
            for i in range(frames)]
    feats = make_features(n, d, seed) if with_features else None
    return Workload(f"panoptic-{n // 1000000}M-1920x1080-D{d}-K8-Q{q}", s, cams, d, 8, feats,
                    make_queries(q, d, seed))
