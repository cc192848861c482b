"""Pins of the oracle's ambiguous-pixel mask: a pixel whose discrete decision
(footprint, alpha >= 1/255, the 0.99 clamp, T < 1e-4) sits exactly at its
threshold must be flagged, with the flag of that decision; a pixel far from
every threshold must not be.  CPU only.  The mask is what lets FP32 results
differ from FP64 ones at such pixels (the blending rule of 3DGS that Sec. 3.2
renders with)."""
import math

import numpy as np

import oracle as _oracle_mod
from paper_2604_12626_gb300 import synth

AMB_VALUE, AMB_COUNT = _oracle_mod.AMB_VALUE, _oracle_mod.AMB_COUNT
AMB_FOOTPRINT, AMB_ALPHA, AMB_STOP, AMB_CLAMP = (_oracle_mod.AMB_FOOTPRINT, _oracle_mod.AMB_ALPHA,
                                                 _oracle_mod.AMB_STOP, _oracle_mod.AMB_CLAMP)
W = H = 64
F = 32.0


def gaussians(xyz, log_sigma, logit):
    n = len(xyz)
    return dict(means=np.array(xyz, np.float32), log_scales=np.full((n, 3), log_sigma, np.float32),
                quats=np.tile(np.float32([1, 0, 0, 0]), (n, 1)), opacity_logits=np.full(n, logit, np.float32),
                sh=np.zeros((n, 16, 3), np.float32))


def camera():
    cam = synth.identity_camera(W, H)
    cam[12:16] = [F, F, (W - 1) / 2, (H - 1) / 2]
    return cam


def s2_of(z, log_sigma):
    return (F * math.exp(float(np.float32(log_sigma))) / z) ** 2 + 0.3


def test_footprint_threshold_is_flagged(oracle):
    # x offset 1/32 m at z = 2 puts the centre at u = 32.0 exactly: pixels 32 +- r
    # lie exactly on the square's edge |i - u| = r
    z, ls = 2.0, -2.0
    g = gaussians([[1.0 / 32.0, 0.0, z]], ls, 2.0)
    out = oracle.render(g, camera(), W, H)
    r = oracle.project(g, camera(), W, H)["radius"][0]
    assert r >= 2
    j = 31  # v = 31.5: row 31 is inside the square
    for i in (32 - r, 32 + r):
        assert out["amb"][j, i] & AMB_FOOTPRINT and out["amb"][j, i] & AMB_COUNT, (i, out["amb"][j, i])
    assert out["amb"][j, 32] & AMB_FOOTPRINT == 0  # the centre column is far from the edge


def test_alpha_threshold_is_flagged(oracle):
    # isotropic, centre at (31.5, 31.5): opacity chosen so that o exp(power) is
    # exactly 1/255 at the pixels 3.5 px out along a row (offset (3.5, 0.5))
    z, ls = 2.0, -1.6
    s2 = s2_of(z, ls)
    d2 = 3.5 ** 2 + 0.5 ** 2
    o = math.exp(0.5 * d2 / s2) / 255.0
    assert 0.0 < o < 0.99
    logit = np.float32(math.log(o / (1.0 - o)))
    g = gaussians([[0.0, 0.0, z]], ls, logit)
    out = oracle.render(g, camera(), W, H)
    o32 = 1.0 / (1.0 + math.exp(-float(logit)))  # the logit is FP32: the threshold moves by ~1e-7
    assert abs(o32 * math.exp(-0.5 * d2 / s2) * 255.0 - 1.0) < 1e-5
    assert out["amb"][31, 35] & AMB_ALPHA and out["amb"][31, 28] & AMB_ALPHA
    assert out["amb"][31, 31] & AMB_ALPHA == 0


def test_clamp_threshold_is_flagged(oracle):
    # a wide splat (sigma 16 px): opacity chosen so that o exp(power) = 0.99
    # exactly at offset (1.5, 0.5)
    z, ls = 2.0, 0.0
    s2 = s2_of(z, ls)
    d2 = 1.5 ** 2 + 0.5 ** 2
    o = 0.99 * math.exp(0.5 * d2 / s2)
    assert 0.99 < o < 1.0
    logit = np.float32(math.log(o / (1.0 - o)))
    g = gaussians([[0.0, 0.0, z]], ls, logit)
    out = oracle.render(g, camera(), W, H)
    assert out["amb"][31, 33] & AMB_CLAMP and out["amb"][31, 30] & AMB_CLAMP
    assert out["amb"][31, 31] & AMB_CLAMP == 0  # clamped well inside the ring
    assert out["amb"][31, 40] & AMB_CLAMP == 0  # well outside it


def test_stop_threshold_is_flagged(oracle):
    # two opaque splats on the axis at 2 m and 3 m: alpha = 0.99 at the centre
    # pixels for both (clamped), so T after the second is 0.01^2 = 1e-4 -- the
    # stop threshold itself
    g = gaussians([[0.0, 0.0, 2.0], [0.0, 0.0, 3.0]], -0.5, 12.0)
    out = oracle.render(g, camera(), W, H)
    assert out["amb"][31, 31] & AMB_STOP and out["amb"][31, 31] & AMB_COUNT
    # a single splat stops nothing and flags no stop
    g1 = gaussians([[0.0, 0.0, 2.0]], -0.5, 12.0)
    assert oracle.render(g1, camera(), W, H)["amb"][31, 31] & AMB_STOP == 0


def test_pixels_far_from_every_threshold_are_not_flagged(oracle):
    g = gaussians([[0.0, 0.0, 3.0]], -1.6, 0.5)  # o = 0.62, no clamp
    out = oracle.render(g, camera(), W, H)
    r = oracle.project(g, camera(), W, H)["radius"][0]
    assert out["amb"][31, 31] == 0 and out["amb"][32, 33] == 0
    assert out["amb"][0, 0] == 0  # uncovered
    assert out["amb"][31, 31 - r + 1] == 0 or out["amb"][31, 31 - r + 1] & AMB_ALPHA  # inside the square
    assert (out["amb"] != 0).mean() < 0.1
