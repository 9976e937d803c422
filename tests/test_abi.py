"""The C ABI library loads and exports every symbol include/psi.h declares;
host-side argument checks (no GPU compute)."""
import ctypes

import pytest

from paper_2604_10982_gb300 import _build, psi


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return psi.lib()


def test_exports_every_declared_symbol(lib):
    names = psi.header_symbols()
    assert len(names) >= 14, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_opts_and_layout(lib):
    o = psi.default_opts()
    assert (o.mode, o.top_k, o.tile_w, o.tile_h) == (psi.EXACT, 0, 16, 16)
    assert abs(o.chi2 - 9.0) < 1e-6 and abs(o.t_eps - 1e-4) < 1e-9
    from paper_2604_10982_gb300 import scenegen as sg
    cams = [sg.look_camera((0, 0, 1.5), 0.0, 150, 100, 100.0), sg.look_camera((0, 0, 1.5), 0.0, 17, 33, 20.0)]
    tb, pb = psi.view_layout(psi.cameras(cams), 2, o)
    assert list(tb) == [0, 10 * 7, 70 + 2 * 3]
    assert list(pb) == [0, 15000, 15000 + 17 * 33]


def test_workspace_sizes(lib):
    assert psi.intersect_workspace_size(0) > 0
    assert psi.sort_workspace_size(10_000) >= 10_000 * 12
    assert psi.render_bwd_workspace_size(1000) >= 1000 * 4
    assert psi.render_bwd_workspace_size(1000, 5000, 8) >= psi.render_bwd_workspace_size(1000) + 5000 * 8 * 4
    assert lib.psi_render_bwd_workspace_size(10, -1, 8, ctypes.byref(ctypes.c_size_t(0))) == psi.PSI_ERR_INVALID_ARG
    b = ctypes.c_size_t(0)
    assert lib.psi_sort_workspace_size(-1, ctypes.byref(b)) == psi.PSI_ERR_INVALID_ARG


def test_null_context_rejected(lib):
    assert lib.psi_project_surfels(None, None, None, 0, None, None, None, None, None) == psi.PSI_ERR_INVALID_ARG
    assert lib.psi_decode_queries(None, None, 0, 128, None, 1, None, None, None, None) == psi.PSI_ERR_INVALID_ARG
    assert lib.psi_last_error(None) == b"NULL context"


def test_ctx_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert lib.psi_ctx_create(ctypes.byref(h), 0) == psi.PSI_ERR_INVALID_ARG
    assert not h.value


def test_time_kernel_rejects_bad_arguments(lib):
    # no context: refused before anything touches a device
    assert lib.psi_ctx_time_kernel(None, psi.KERNEL_BWD_WALK, None, None) == psi.PSI_ERR_INVALID_ARG


def test_render_shape_calls_check_arguments(lib):
    """The launch-shape calls refuse a missing context before touching a GPU."""
    o = psi.default_opts(top_k=8)
    v = ctypes.c_int(-1)
    assert lib.psi_ctx_set_render_shape(None, 0, ctypes.byref(o), psi.F32, 0, 1) == psi.PSI_ERR_INVALID_ARG
    assert lib.psi_ctx_get_render_shape(None, 1, ctypes.byref(o), psi.F32, 1, ctypes.byref(v)) == psi.PSI_ERR_INVALID_ARG
    assert psi.RENDER_SHAPES == 16


def test_context_creation_without_a_device_fails_cleanly(lib):
    """On a machine without a CUDA device the library still loads and a
    context request returns an error code instead of crashing."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    h = ctypes.c_void_p(None)
    rc = lib.psi_ctx_create(ctypes.byref(h), 0)
    assert rc == psi.PSI_ERR_INVALID_ARG and not h.value  # device 0 does not exist
