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


def test_tiny_config_shape(oracle_lib):
    w = sg.tiny()
    assert w.surfels.n == 2000 and w.cameras[0].width == 128 and w.features.shape == (2000, 16)
    out = orc.render(w.surfels, w.cameras[0], orc.Opts(top_k=8), feat=w.features)
    assert np.max(np.abs(out["sumw"] + out["T"] - 1.0)) < 1e-12


@pytest.mark.parametrize("plant,check", [
    (1, "fronto"), (2, "two"), (3, "topk"), (4, "fd"), (5, "coverage"),
])
def test_planted_mistake_is_caught(plant, check):
    """A deliberately wrong oracle build fails the pin aimed at that mistake."""
    fn = {
        "fronto": pins.pin_fronto_parallel,
        "two": pins.pin_two_surfels,
        "topk": lambda: pins.pin_topk_special_cases(sg.dense_box(n=3000)),
        "fd": lambda: pins.fd_check(sg.crop_scene(n=200, d=8, size=48), params_per_kind=6),
        "coverage": lambda: pins.pin_coverage(sg.dense_box(n=3000), modes=(orc.EXACT,)),
    }[check]
    orc.use_variant(plant)
    try:
        with pytest.raises(AssertionError):
            fn()
    finally:
        orc.use_variant(0)
