"""Pins of the oracle's FP32 error bounds (the ambiguity mask's inputs) against
an independent single-precision evaluation of the projection: the quantities
the CUDA path takes its decisions on -- the screen position (u, v), the radius
term 3 sqrt(lambda) and the conic (A, B, C) -- evaluated here with numpy float32
operations (every operation correctly rounded) in the order of the standard
EWA definitions, must lie within the oracle's bound of its FP64 value for every
Gaussian, and the bounds must not be vacuous.  CPU only."""
import numpy as np

from paper_2604_12626_gb300 import synth

f32 = np.float32


def _fp32_projection(g, cam, W, H):
    """(u - cx, v - cy, 3 sqrt(lambda), A, B, C) in float32, per Gaussian: the
    2D covariance of a scale-rotation Gaussian from its factor G = T R diag(e^s),
    the determinant as 0.3 tr + 0.09 plus the squared minors of G."""
    cam = cam.astype(f32)
    R = cam[:9].reshape(3, 3)
    C = cam[9:12]
    fx, fy = cam[12], cam[13]
    mu = g["means"].astype(f32)
    d = mu - C
    p = np.stack([d[:, 0] * R[r, 0] + d[:, 1] * R[r, 1] + d[:, 2] * R[r, 2] for r in range(3)], 1).astype(f32)
    px, py, pz = p[:, 0], p[:, 1], p[:, 2]
    tx, ty = px / pz, py / pz
    uc, vc = fx * tx, fy * ty
    limx = f32(1.3) * (f32(0.5) * f32(W) / fx)
    limy = f32(1.3) * (f32(0.5) * f32(H) / fy)
    txc, tyc = np.clip(tx, -limx, limx), np.clip(ty, -limy, limy)
    j00, j02 = fx / pz, -(fx * txc) / pz
    j11, j12 = fy / pz, -(fy * tyc) / pz
    t0 = np.stack([j00 * R[0, c] + j02 * R[2, c] for c in range(3)], 1)
    t1 = np.stack([j11 * R[1, c] + j12 * R[2, c] for c in range(3)], 1)
    # Sigma = (R(q) diag(exp s)) (R(q) diag(exp s))^T
    q = g["quats"].astype(f32)
    inv = f32(1) / np.sqrt(q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1] + q[:, 2] * q[:, 2] + q[:, 3] * q[:, 3])
    w, x, y, z = (q[:, i] * inv for i in range(4))
    two = f32(2)
    Rq = np.stack([f32(1) - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y),
                   two * (x * y + w * z), f32(1) - two * (x * x + z * z), two * (y * z - w * x),
                   two * (x * z - w * y), two * (y * z + w * x), f32(1) - two * (x * x + y * y)], 1).reshape(-1, 3, 3)
    # exp correctly rounded to float32 (the bound assumes at most 2 ulp)
    sc = np.exp(g["log_scales"].astype(f32).astype(np.float64)).astype(f32)
    M = Rq * sc[:, None, :]
    # G = T M; Sigma2 = G G^T + 0.3 I; det by the squared 2 x 2 minors of G
    G0 = sum(t0[:, k, None] * M[:, k, :] for k in range(3)).astype(f32)
    G1 = sum(t1[:, k, None] * M[:, k, :] for k in range(3)).astype(f32)
    a1 = G0[:, 0] * G0[:, 0] + G0[:, 1] * G0[:, 1] + G0[:, 2] * G0[:, 2]
    c1 = G1[:, 0] * G1[:, 0] + G1[:, 1] * G1[:, 1] + G1[:, 2] * G1[:, 2]
    b = G0[:, 0] * G1[:, 0] + G0[:, 1] * G1[:, 1] + G0[:, 2] * G1[:, 2]
    m01 = G0[:, 0] * G1[:, 1] - G0[:, 1] * G1[:, 0]
    m02 = G0[:, 0] * G1[:, 2] - G0[:, 2] * G1[:, 0]
    m12 = G0[:, 1] * G1[:, 2] - G0[:, 2] * G1[:, 1]
    dg = m01 * m01 + m02 * m02 + m12 * m12
    a, c = a1 + f32(0.3), c1 + f32(0.3)
    det = f32(0.3) * (a1 + c1) + dg + f32(0.3) * f32(0.3)
    mid = f32(0.5) * (a + c)
    hd = f32(0.5) * (a - c)
    lam = mid + np.sqrt(np.maximum(f32(0.1), hd * hd + b * b))
    r3 = f32(3) * np.sqrt(lam)
    idet = f32(1) / det
    return uc, vc, r3, c * idet, -b * idet, a * idet


def _scenes():
    rng = np.random.default_rng(7)
    W, H = 256, 192
    room = synth.room_scene(20_000, seed=3)
    yield room, synth.room_camera(3, W, H), W, H
    # near-isotropic Gaussians of a few to tens of pixels, the discriminant just
    # above its 0.1 floor (cancellation in mid^2 - det), and very flat ones
    n = 6000
    g = synth.box_scene(n, seed=5)
    base = rng.uniform(-4.5, -2.0, n)
    ls = np.stack([base, base + rng.uniform(0, 0.05, n), base + rng.uniform(0, 0.05, n)], 1)
    flat = rng.random(n) < 0.3
    ls[flat, 2] -= 4.0
    g["log_scales"] = ls.astype(np.float32)
    yield g, synth.identity_camera(W, H), W, H
    # large, nearly isotropic Gaussians (tens of px^2, anisotropy of 0.1-0.3%):
    # mid^2 - det cancels down to a discriminant just above the floor
    g = synth.box_scene(n, seed=6)
    base = rng.uniform(-1.5, -0.8, n)
    ls = np.stack([base, base + rng.uniform(0, 0.003, n), base + rng.uniform(0, 0.003, n)], 1)
    g["log_scales"] = ls.astype(np.float32)
    yield g, synth.identity_camera(W, H), W, H
    # needles (one long axis): the 2D covariance nearly singular before the
    # dilation, a c / det in the hundreds (the determinant's own rounding)
    g = synth.box_scene(n, seed=7)
    ls = np.stack([rng.uniform(-2.0, -0.5, n), np.full(n, -8.0), np.full(n, -8.0)], 1)
    g["log_scales"] = ls.astype(np.float32)
    yield g, synth.identity_camera(W, H), W, H


def test_fp32_projection_within_the_oracle_bounds(oracle):
    worst = np.zeros(6)
    for g, cam, W, H in _scenes():
        pr = oracle.project(g, cam, W, H)
        sel = (pr["z"] > 0.2) & (pr["r3"] > 0)
        cam64 = cam.astype(np.float32).astype(np.float64)
        got = [np.asarray(x, np.float64)[sel] for x in _fp32_projection(g, cam, W, H)]
        ref = [pr["u"][sel] - cam64[14], pr["v"][sel] - cam64[15], pr["r3"][sel],
               pr["conic"][sel, 0], pr["conic"][sel, 1], pr["conic"][sel, 2]]
        bnd = [pr["err_uv"][sel, 0], pr["err_uv"][sel, 1], pr["err_r3"][sel],
               pr["err_conic"][sel, 0], pr["err_conic"][sel, 1], pr["err_conic"][sel, 2]]
        for k, (x, r, e) in enumerate(zip(got, ref, bnd)):
            ok = np.isfinite(x)
            over = np.abs(x - r)[ok] > e[ok]
            assert not over.any(), (k, np.flatnonzero(over)[:5], (np.abs(x - r)[ok] / e[ok]).max())
            worst[k] = max(worst[k], (np.abs(x - r)[ok] / np.maximum(e[ok], 1e-300)).max())
    # first-order worst cases: the realized FP32 errors reach a visible share of them
    assert (worst > 0.02).all(), worst
