"""The oracle's FP64 adjoint against FP64 central finite differences of the
oracle's forward (render, and LBS feeding render).  CPU only.

Loss L = <w_rgb, rgb> + <w_d, depth> with fixed random weights.  A coordinate
is discarded when FD(h) and FD(h/2) disagree (a discrete decision straddled).
"""
import numpy as np
import pytest

from fd_case import W, H, as64, central_differences, fd_camera, fd_scene, loss_and_pieces
from paper_2604_12626_gb300 import synth


def test_adjoint_matches_finite_differences(oracle):
    sc, av, G = fd_scene()
    sc, av = as64(sc), as64(av)
    cam = fd_camera()
    rng = np.random.default_rng(1)
    wr = rng.standard_normal((3, H, W))
    wd = rng.standard_normal((H, W))
    L0, g, out = loss_and_pieces(oracle, sc, av, G, cam, wr, wd)
    assert (out["T"] < 0.9).mean() > 0.2
    pr = oracle.project(g, cam, W, H)
    jj, ii = np.mgrid[0:H, 0:W]
    clamped = 0
    for k in np.flatnonzero(pr["visible"] & (pr["opacity"] > 0.99)):
        A, B, C = pr["conic"][k]
        dx, dy = pr["u"][k] - ii, pr["v"][k] - jj
        clamped += int((pr["opacity"][k] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy) > 0.99).sum())
    assert clamped >= 5  # the 0.99 clamp is exercised
    n_s = len(sc["means"])
    gr = oracle.render_backward(g, cam, W, H, wr, wd)
    ga = oracle.lbs_backward(av["means"], av["log_scales"], av["quats"], av["joint_ids"], av["weights"],
                             np.zeros(len(av["means"]), np.int32), G, gr["means"][n_s:], gr["cov3d"][n_s:])
    analytic = {
        ("sc", "means"): gr["means"][:n_s], ("sc", "log_scales"): gr["log_scales"][:n_s],
        ("sc", "quats"): gr["quats"][:n_s], ("sc", "opacity_logits"): gr["opacity_logits"][:n_s],
        ("sc", "sh"): gr["sh"][:n_s], ("av", "means"): ga["means"], ("av", "log_scales"): ga["log_scales"],
        ("av", "quats"): ga["quats"], ("av", "opacity_logits"): gr["opacity_logits"][n_s:],
        ("av", "sh"): gr["sh"][n_s:], ("G", "G"): ga["G"],
    }
    checked = 0
    for (owner, key), A in analytic.items():
        base = {"sc": sc, "av": av, "G": {"G": G}}[owner][key]
        flat_idx = rng.choice(base.size, size=min(base.size, 40), replace=False)
        kept, refs = central_differences(oracle, sc, av, G, cam, wr, wd, owner, key, flat_idx)
        assert len(refs) >= 20, (owner, key)
        errs = A.ravel()[kept] - refs
        scale = np.abs(refs).max() + 1e-12
        assert np.abs(errs).max() <= 1e-5 * scale + 5e-8, (owner, key, np.abs(errs).max(), scale)
        checked += len(refs)
    assert checked > 300


def test_lbs_adjoint_matches_finite_differences(oracle):
    av = as64(synth.avatar_canonical(30, 3))
    rng = np.random.default_rng(2)
    G = rng.normal(0, 0.5, (2, 24, 3, 4))
    avatar_of = (np.arange(30) % 2).astype(np.int32)
    wm = rng.standard_normal((30, 3))
    wc = rng.standard_normal((30, 6))

    def L():
        m, c = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"], av["weights"], avatar_of, G)
        return float((wm * m).sum() + (wc * c).sum())

    ga = oracle.lbs_backward(av["means"], av["log_scales"], av["quats"], av["joint_ids"], av["weights"], avatar_of,
                             G, wm, wc)
    for arr, grad in [(av["means"], ga["means"]), (av["log_scales"], ga["log_scales"]), (av["quats"], ga["quats"]),
                      (G, ga["G"])]:
        for fi in rng.choice(arr.size, size=25, replace=False):
            idx = np.unravel_index(fi, arr.shape)
            x0 = arr[idx]
            h = 1e-6 * max(abs(x0), 1.0)
            arr[idx] = x0 + h
            Lp = L()
            arr[idx] = x0 - h
            Lm = L()
            arr[idx] = x0
            assert grad[idx] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6, abs=1e-9)
