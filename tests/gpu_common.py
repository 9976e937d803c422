"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc
from paper_2604_10982_gb300 import scenegen as sg

# Excusal rules for FP32-vs-FP64 value comparisons.
#  - straddle: some surfel's u^2+v^2 is within 1e-5 (relative) of r^2, its alpha
#    within 1e-5 of 1/255, or T within 1e-5 of T_eps at a compositing step: the
#    two precisions may take the other branch there;
#  - ill-conditioned: one unit in the last place of the image coordinate
#    (2^-24 * max(W, H) pixels) moves the pixel's value by more than the 1e-4
#    tolerance (diag[4] is the oracle's d(value)/d(pixel position));
#  - near tie: the K-th and (K+1)-th Top-K weights differ by <= 1e-6.
# Excused pixels are counted, and still checked against a gross-error bound.
STRADDLE = 1e-5
COND_TOL = 1e-4
NEAR_TIE = 1e-6
GROSS = 5e-2


def opts_of(o: "orc.Opts"):
    from paper_2604_10982_gb300 import psi
    return psi.default_opts(mode=o.mode, top_k=o.top_k, chi2=o.chi2, z_near=o.z_near,
                            opacity_radius=int(o.opacity_radius), tile_w=o.tile_w, tile_h=o.tile_h, t_eps=o.t_eps)


def flags(out, cam):
    """Per-pixel excusal masks from the oracle's diagnostics."""
    d = out["diag"]
    dp = 2.0 ** -24 * max(cam.width, cam.height)
    straddle = (d[:, 0] < STRADDLE) | (d[:, 1] < STRADDLE) | (d[:, 2] < STRADDLE)
    illcond = d[:, 4] * dp > COND_TOL
    neartie = d[:, 3] < NEAR_TIE
    return straddle, illcond, neartie


def multi_cams():
    return [sg.look_camera((0.0, -6.0, 1.5), 0.0, 150, 100, 129.0),
            sg.look_camera((0.7, -5.5, 1.2), 0.25, 77, 45, 60.0),
            sg.look_camera((-0.5, -6.5, 2.0), -0.2, 128, 128, 110.0)]
