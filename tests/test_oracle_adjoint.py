"""The oracle's FP64 adjoint against FP64 central finite differences of the
oracle's forward (render, and LBS feeding render).  CPU only.

Loss L = <w_rgb, rgb> + <w_d, depth> with fixed random weights.  A coordinate
is discarded when FD(h) and FD(h/2) disagree (a discrete decision straddled).
"""
import numpy as np
import pytest

from paper_2604_12626_gb300 import synth

W = H = 32
F = 16.0


def fd_scene(seed=0, n_scene=100, n_av=100):
    """100 scene Gaussians in view plus 100 avatar Gaussians posed in view."""
    rng = np.random.default_rng(seed)
    sc = synth.box_scene(n_scene, seed=seed)
    sc["means"][:, :2] *= 0.8
    sc["means"][:, 2] = rng.uniform(2.0, 5.0, n_scene).astype(np.float32)
    sc["log_scales"] = rng.normal(-1.3, 0.3, (n_scene, 3)).astype(np.float32)
    sc["sh"][:, 1:, :] = rng.normal(0, 0.2, (n_scene, 15, 3)).astype(np.float32)
    # every 4th: large and nearly opaque, so that alpha is clamped at 0.99 near its centre
    sc["opacity_logits"][::4] = rng.uniform(8.0, 10.0, len(sc["opacity_logits"][::4]))
    sc["log_scales"][::4] += np.float32(1.0)
    av = synth.avatar_canonical(n_av, seed)
    av["means"] *= np.float32(0.4)
    av["log_scales"] = rng.normal(-2.0, 0.3, (n_av, 3)).astype(np.float32)
    G = np.zeros((1, 24, 3, 4))
    for j in range(24):
        from scipy.spatial.transform import Rotation
        G[0, j, :, :3] = Rotation.from_rotvec(rng.normal(0, 0.15, 3)).as_matrix()
        G[0, j, :, 3] = [0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(), 3.0]
    return sc, av, G


def loss_and_pieces(oracle, sc, av, G, cam, wr, wd):
    m, c = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"], av["weights"],
                      np.zeros(len(av["means"]), np.int32), G)
    n_s = len(sc["means"])
    g = dict(means=np.concatenate([np.asarray(sc["means"], np.float64), m]),
             log_scales=np.concatenate([sc["log_scales"], av["log_scales"]]).astype(np.float64),
             quats=np.concatenate([sc["quats"], av["quats"]]).astype(np.float64),
             opacity_logits=np.concatenate([sc["opacity_logits"], av["opacity_logits"]]).astype(np.float64),
             sh=np.concatenate([sc["sh"], av["sh"]]).astype(np.float64),
             cov3d=np.concatenate([np.zeros((n_s, 6)), c]),
             use_cov=np.concatenate([np.zeros(n_s, np.uint8), np.ones(len(m), np.uint8)]))
    out = oracle.render(g, cam, W, H, nthreads=1)
    L = float((wr * out["rgb"]).sum() + (wd * out["depth"]).sum())
    return L, g, out


def as64(d):
    return {k: (np.array(v, np.float64) if k not in ("joint_ids",) else v) for k, v in d.items()}


def test_adjoint_matches_finite_differences(oracle):
    sc, av, G = fd_scene()
    sc, av = as64(sc), as64(av)
    cam = synth.identity_camera(W, H)
    cam[12:14] = F
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
        src = {"sc": sc, "av": av, "G": {"G": G}}[owner]
        base = src[key]
        flat_idx = rng.choice(base.size, size=min(base.size, 40), replace=False)
        errs, refs = [], []
        for fi in flat_idx:
            idx = np.unravel_index(fi, base.shape)
            x0 = base[idx]
            fds = []
            for h in (1e-6 * max(abs(x0), 1.0), 0.5e-6 * max(abs(x0), 1.0)):
                base[idx] = x0 + h
                Lp = loss_and_pieces(oracle, sc, av, G, cam, wr, wd)[0]
                base[idx] = x0 - h
                Lm = loss_and_pieces(oracle, sc, av, G, cam, wr, wd)[0]
                base[idx] = x0
                fds.append((Lp - Lm) / (2 * h))
            if abs(fds[0] - fds[1]) > 1e-3 * max(abs(fds[0]), 1e-6):
                continue  # a threshold was straddled
            errs.append(A[idx] - fds[0])
            refs.append(fds[0])
        refs = np.array(refs)
        errs = np.array(errs)
        assert len(refs) >= 20, (owner, key)
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
