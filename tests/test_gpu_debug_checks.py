"""The bounds-checked debug build (needs a GPU).

libpsi_debug.so is the library compiled with PSI_DEBUG: every index the
pipeline kernels take from data -- the tile launch order, the tile ranges, the
record index of each list entry, the surfel ids of selected slots and of the
caller's saved Top-K set -- is checked against its buffer before use; a
failure raises PSI_ERR_BOUNDS with the check site and the access is clamped to
a valid index. compute-sanitizer is closed on this machine, so this build is the
check of those indices: the parity suites run against it in a child process
(every one of their status checks must stay clean), and corrupted inputs,
which the release build would turn into out-of-range reads, are caught there.
The corruption tests run only when the debug library is the one loaded."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

from .gpu_common import multi_cams, opts_of

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _debug_loaded():
    from paper_2604_10982_gb300 import psi
    return psi.lib().psi_debug_checks() == 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_10982_gb300 import psi
    return psi.Context(0)


def test_parity_suites_clean_under_the_debug_build(ctx):
    """The parity, gradient and tile suites with libpsi_debug.so, plus the
    corruption tests of this file, in a child process."""
    if _debug_loaded():
        pytest.skip("this process already runs the debug build")
    from paper_2604_10982_gb300 import _build
    _build.build(debug=True)
    env = dict(os.environ, PSI_LIBRARY="debug")
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_grad.py", "tests/test_gpu_tiles.py",
             "tests/test_gpu_debug_checks.py"]
    r = subprocess.run([sys.executable, "-m", "pytest", *files, "-m", "gpu", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert "passed" in tail and "skipped" in tail  # the first test of this file skips itself there


def _frame(ctx, K=8):
    from paper_2604_10982_gb300 import pipeline as pl, psi
    w = sg.dense_box(n=3000, d=32)
    cams = multi_cams()
    o = orc.Opts(mode=orc.EXACT, top_k=K, opacity_radius=True)
    scene = pl.DeviceScene(w.surfels, w.features, feat_dtype=psi.BF16)
    r = pl.make_renderer(ctx, scene, cams, opts_of(o), D=32)
    r.frame(scene)
    torch.cuda.synchronize()
    assert ctx.status_fetch() == (0, 0)
    return w, scene, r


def test_bad_saved_topk_id_is_caught(ctx):
    """A saved Top-K id past the surfel table reaching the adjoint."""
    if not _debug_loaded():
        pytest.skip("needs the debug build (runs in the child process of the test above)")
    from paper_2604_10982_gb300 import psi
    w, scene, r = _frame(ctx)
    r.topk_ids.view(-1)[1234] = scene.n + 5
    P = r.n_pix
    gC = torch.ones(3, P, device="cuda")
    gF = torch.ones(P, 32, device="cuda")
    r.backward(scene, gC, gF)
    st, site = ctx.status_fetch()
    assert st == psi.PSI_ERR_BOUNDS and site == 104, (st, site)


def test_bad_launch_order_is_caught(ctx):
    """An entry of the compositing launch order past the frame's tiles."""
    if not _debug_loaded():
        pytest.skip("needs the debug build (runs in the child process of the test above)")
    from paper_2604_10982_gb300 import psi
    w, scene, r = _frame(ctx)
    r.ranges[2 * r.n_tiles + 3] = r.n_tiles + 7
    r.render(scene)
    st, site = ctx.status_fetch()
    assert st == psi.PSI_ERR_BOUNDS and site == 101, (st, site)


def test_bad_list_entry_is_caught(ctx):
    """A list entry naming a record outside the tile's view (the multi-view
    frame: records of another view are valid memory but the wrong surfel)."""
    if not _debug_loaded():
        pytest.skip("needs the debug build (runs in the child process of the test above)")
    from paper_2604_10982_gb300 import psi
    w, scene, r = _frame(ctx)
    rg = r.ranges[: 2 * r.n_tiles].view(-1, 2).cpu().numpy().view(np.uint32).astype(np.int64)
    # the first view's tiles hold records [0, N); make one entry name a record of the last view
    t = int(np.argmax((rg[:, 1] - rg[:, 0])[: int(r.tile_base[1])]))
    assert rg[t, 1] > rg[t, 0]
    r.vals[int(rg[t, 0])] = 2 * scene.n + 1
    r.render(scene)
    st, site = ctx.status_fetch()
    assert st == psi.PSI_ERR_BOUNDS and site == 103, (st, site)


def test_bad_saved_last_position_is_caught(ctx):
    """A saved last-composited position past the end of its tile's list (it
    bounds the adjoint's reverse walk)."""
    if not _debug_loaded():
        pytest.skip("needs the debug build (runs in the child process of the test above)")
    from paper_2604_10982_gb300 import psi
    w, scene, r = _frame(ctx)
    r.n_last.view(-1)[777] = 1 << 20
    P = r.n_pix
    gC = torch.ones(3, P, device="cuda")
    gF = torch.ones(P, 32, device="cuda")
    r.backward(scene, gC, gF)
    st, site = ctx.status_fetch()
    assert st == psi.PSI_ERR_BOUNDS and site == 105, (st, site)
