"""The finite-difference case of the adjoint tests: 100 scene Gaussians and one
100-Gaussian avatar (24 joints) posed by LBS, all in view of one 32x32 camera
with f = 16, and the FP64 oracle loss L = <w_rgb, rgb> + <w_d, depth> of the
scene plus posed avatar rendered in one pass.  Shared by the oracle's own FD
test (CPU) and the CUDA adjoint's FD test (GPU)."""
import numpy as np
from scipy.spatial.transform import Rotation

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
        G[0, j, :, :3] = Rotation.from_rotvec(rng.normal(0, 0.15, 3)).as_matrix()
        G[0, j, :, 3] = [0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(), 3.0]
    return sc, av, G


def fd_camera():
    cam = synth.identity_camera(W, H)
    cam[12:14] = F
    return cam


def posed_scene(oracle, sc, av, G):
    """The oracle's input for scene + avatar: LBS in FP64, posed rows by covariance."""
    m, c = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"], av["weights"],
                      np.zeros(len(av["means"]), np.int32), G)
    n_s = len(sc["means"])
    return dict(means=np.concatenate([np.asarray(sc["means"], np.float64), m]),
                log_scales=np.concatenate([sc["log_scales"], av["log_scales"]]).astype(np.float64),
                quats=np.concatenate([sc["quats"], av["quats"]]).astype(np.float64),
                opacity_logits=np.concatenate([sc["opacity_logits"], av["opacity_logits"]]).astype(np.float64),
                sh=np.concatenate([sc["sh"], av["sh"]]).astype(np.float64),
                cov3d=np.concatenate([np.zeros((n_s, 6)), c]),
                use_cov=np.concatenate([np.zeros(n_s, np.uint8), np.ones(len(m), np.uint8)]))


def loss_and_pieces(oracle, sc, av, G, cam, wr, wd):
    g = posed_scene(oracle, sc, av, G)
    out = oracle.render(g, cam, W, H, nthreads=1)
    L = float((wr * out["rgb"]).sum() + (wd * out["depth"]).sum())
    return L, g, out


def as64(d):
    return {k: (np.array(v, np.float64) if k not in ("joint_ids",) else v) for k, v in d.items()}


def central_differences(oracle, sc, av, G, cam, wr, wd, owner, key, flat_idx, h_rel=1e-6):
    """FP64 central differences of L at the given flat indices of one input
    array, with step h = h_rel max(|x|, 1) and h / 2; a coordinate whose two
    estimates disagree by more than 1e-3 (relative) straddles a discrete
    decision and is dropped.  Returns (kept flat indices, FD values)."""
    base = {"sc": sc, "av": av, "G": {"G": G}}[owner][key]
    kept, vals = [], []
    for fi in flat_idx:
        idx = np.unravel_index(fi, base.shape)
        x0 = base[idx]
        fds = []
        for h in (h_rel * max(abs(x0), 1.0), 0.5 * h_rel * max(abs(x0), 1.0)):
            base[idx] = x0 + h
            Lp = loss_and_pieces(oracle, sc, av, G, cam, wr, wd)[0]
            base[idx] = x0 - h
            Lm = loss_and_pieces(oracle, sc, av, G, cam, wr, wd)[0]
            base[idx] = x0
            fds.append((Lp - Lm) / (2 * h))
        if abs(fds[0] - fds[1]) > 1e-3 * max(abs(fds[0]), 1e-6):
            continue
        kept.append(int(fi))
        vals.append(fds[0])
    return np.array(kept, np.int64), np.array(vals)
