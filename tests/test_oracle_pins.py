"""Pins of the FP64 oracle to facts outside itself: closed forms, symmetries,
invariants, library routines (scipy) and finite differences.  CPU only.

Each test names the part of the rendering definition it pins (3DGS
rasterisation as cited in Sec. 2.2 / Sec. 3.2; LBS as in Sec. 3.3).  A
plausible slip in the oracle -- a dropped dilation, a transposed rotation, a
wrong SH sign, a skipped clamp, an off-by-one in the stop rule -- fails at
least one of them (see ``test_planted_mistakes_are_caught``).
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2604_12626_gb300 import synth

C0 = 0.5 / math.sqrt(math.pi)  # sqrt(1 / (4 pi))


def one_gaussian(z, log_sigma, logit, k0, quat=(1.0, 0.0, 0.0, 0.0), xy=(0.0, 0.0)):
    return dict(
        means=np.array([[xy[0], xy[1], z]], np.float32),
        log_scales=np.full((1, 3), log_sigma, np.float32),
        quats=np.array([quat], np.float32),
        opacity_logits=np.array([logit], np.float32),
        sh=np.concatenate([np.array(k0, np.float32).reshape(1, 1, 3), np.zeros((1, 15, 3), np.float32)], 1),
    )


def cam_f(W, H, f, cx=None, cy=None):
    cam = synth.identity_camera(W, H)
    cam[12:16] = [f, f, (W - 1) / 2 if cx is None else cx, (H - 1) / 2 if cy is None else cy]
    return cam


# ---------------------------------------------------------------------------
# closed form: one isotropic Gaussian on the optical axis
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("z,ls,logit,f", [(3.0, -2.5, 0.3, 16.5), (2.0, -3.0, 5.0, 24.0), (5.0, -1.5, -1.0, 16.0)])
def test_single_gaussian_closed_form(oracle, z, ls, logit, f):
    W = H = 33
    k0 = [0.4, -0.2, 1.1]
    g = one_gaussian(z, ls, logit, k0)
    cam = cam_f(W, H, f)
    out = oracle.render(g, cam, W, H, mode="pixel")
    sigma = math.exp(float(np.float32(ls)))
    s2 = (f * sigma / z) ** 2 + 0.3  # J Sigma J^T + dilation, isotropic
    r = math.ceil(3.0 * math.sqrt(s2 + math.sqrt(0.1)))
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    col = np.maximum(0.0, C0 * np.float32(k0).astype(np.float64) + 0.5)
    c = (W - 1) / 2
    jj, ii = np.mgrid[0:H, 0:W].astype(np.float64)
    rho2 = (ii - c) ** 2 + (jj - c) ** 2
    alpha = np.minimum(0.99, o * np.exp(-0.5 * rho2 / s2))
    covered = np.maximum(np.abs(ii - c), np.abs(jj - c)) <= r
    blended = covered & (alpha >= 1.0 / 255.0)
    a = np.where(blended, alpha, 0.0)
    np.testing.assert_allclose(out["rgb"], col[:, None, None] * a[None], rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["T"], 1.0 - a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["depth"], z * a, rtol=0, atol=1e-12)
    assert np.array_equal(out["n_contrib"], blended.astype(np.int32))
    assert out["evals"] == int(covered.sum())  # one examination per covered pixel
    assert oracle.project(g, cam, W, H)["radius"][0] == r  # 0.1 floor on the discriminant
    if logit >= 5.0:
        assert abs(out["T"][int(c), int(c)] - 0.01) < 1e-15  # 0.99 clamp at the centre


def test_elongated_gaussian_square_footprint_closed_form(oracle):
    # axis-aligned ellipse: Sigma2 = diag(a, c); r = ceil(3 sqrt(max(a, c))).  The
    # x semi-axis is chosen so that 3 sqrt(a) sits just below 10: the pixel 11 px
    # out on the axis still has alpha >= 1/255 but lies outside the square.
    W = H = 33
    f, z = 16.0, 2.0
    lsx = np.float32(0.5 * math.log((11.1 - 0.3) / 64.0))
    g = one_gaussian(z, -3.0, 4.6, [0.3, 0.3, 0.3])
    g["log_scales"][0, 0] = lsx
    cam = cam_f(W, H, f)
    out = oracle.render(g, cam, W, H, mode="pixel")
    a = (f * math.exp(float(lsx)) / z) ** 2 + 0.3
    c = (f * math.exp(-3.0) / z) ** 2 + 0.3
    assert ((a + c) / 2) ** 2 - a * c >= 0.1
    r = math.ceil(3 * math.sqrt(max(a, c)))
    assert r == 10
    o = 1 / (1 + math.exp(-float(np.float32(4.6))))
    col = C0 * np.float32(0.3) + 0.5
    jj, ii = np.mgrid[0:H, 0:W].astype(np.float64)
    dx, dy = ii - 16, jj - 16
    alpha = np.minimum(0.99, o * np.exp(-0.5 * (dx * dx / a + dy * dy / c)))
    covered = np.maximum(np.abs(dx), np.abs(dy)) <= r
    assert alpha[16, 16 + r + 1] >= 1 / 255  # the cut is visible
    blended = covered & (alpha >= 1 / 255)
    np.testing.assert_allclose(out["rgb"][0], col * np.where(blended, alpha, 0.0), atol=1e-13)
    assert out["rgb"][0][16, 16 + r + 1] == 0.0
    assert oracle.project(g, cam, W, H)["radius"][0] == r


def test_background_and_normalised_depth(oracle):
    W = H = 17
    g = one_gaussian(2.5, -2.0, 0.5, [0.1, 0.2, 0.3])
    cam = cam_f(W, H, 12.0)
    bg = (0.25, 0.5, 0.75)
    a = oracle.render(g, cam, W, H, bg=bg)
    b = oracle.render(g, cam, W, H)
    np.testing.assert_allclose(a["rgb"] - b["rgb"], np.array(bg)[:, None, None] * b["T"][None], atol=1e-15)
    n = oracle.render(g, cam, W, H, normalize_depth=True)
    on = (1.0 - b["T"]) >= 1e-4
    np.testing.assert_allclose(n["depth"][on], 2.5, rtol=1e-12)
    assert np.all(n["depth"][~on] == 0.0)


# ---------------------------------------------------------------------------
# symmetry of isotropic splats on the axis; pixel centres at integer coords
# ---------------------------------------------------------------------------
def test_isotropic_symmetry(oracle):
    W = H = 32
    gs = [one_gaussian(z, ls, lg, k0) for z, ls, lg, k0 in
          [(2.0, -2.8, 0.2, [0.3, -0.1, 0.5]), (3.0, -2.0, -0.5, [-0.4, 0.6, 0.1]), (4.5, -1.7, 1.5, [0.9, 0.2, -0.3])]]
    g = {k: np.concatenate([x[k] for x in gs]) for k in gs[0]}
    out = oracle.render(g, cam_f(W, H, 16.0), W, H, mode="pixel")
    for key in ("rgb", "depth", "T", "n_contrib"):
        im = out[key]
        assert np.array_equal(im, im[..., ::-1]), key
        assert np.array_equal(im, im[..., ::-1, :]), key
        assert np.array_equal(im, np.swapaxes(im, -1, -2)), key


# ---------------------------------------------------------------------------
# transmittance product: rgb = 1 - T for white Gaussians, depth = z (1 - T)
# ---------------------------------------------------------------------------
def test_transmittance_invariant(oracle):
    g = synth.box_scene(3000, seed=3)
    g["sh"][:] = 0.0
    g["sh"][:, 0, :] = np.float32(0.5 / C0)
    g["means"][:, 2] = np.float32(4.0)
    g["log_scales"] += np.float32(2.5)
    W = H = 96
    cam = cam_f(W, H, 48.0)
    out = oracle.render(g, cam, W, H)
    assert (out["T"] < 0.5).mean() > 0.2  # the invariant is exercised on covered pixels
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], 1.0 - out["T"], atol=1e-12)
    np.testing.assert_allclose(out["depth"], 4.0 * (1.0 - out["T"]), atol=1e-11)
    assert out["T"].min() >= 1e-4  # blending never takes T below the stop level


def test_stop_rule_never_blends_below_threshold(oracle):
    # 40 opaque white splats stacked on the axis: the pixel stops before T < 1e-4
    n = 40
    g = dict(means=np.stack([np.zeros(n), np.zeros(n), np.linspace(2, 4, n)], 1).astype(np.float32),
             log_scales=np.full((n, 3), -2.0, np.float32), quats=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
             opacity_logits=np.full(n, 3.0, np.float32), sh=np.zeros((n, 16, 3), np.float32))
    W = H = 9
    out = oracle.render(g, cam_f(W, H, 8.0), W, H)
    o = 1 / (1 + math.exp(-3.0))
    # centre: T_k = (1-o)^k; blending stops before the first k with T_k < 1e-4
    k_stop = next(k for k in range(1, n) if (1 - o) ** k < 1e-4)
    assert out["n_contrib"][4, 4] == k_stop - 1
    assert abs(out["T"][4, 4] - (1 - o) ** (k_stop - 1)) < 1e-15


def test_evaluation_count_closed_form(oracle):
    # 30 wide isotropic splats stacked on the axis, each covering the whole 9x9
    # image: per pixel, the examinations are the splats in depth order up to and
    # including the first whose blend would take T below 1e-4 (or all of them)
    n, W, f, o = 30, 9, 8.0, 0.9
    z = np.linspace(2.0, 4.0, n)
    g = dict(means=np.stack([np.zeros(n), np.zeros(n), z], 1).astype(np.float32),
             log_scales=np.zeros((n, 3), np.float32), quats=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
             opacity_logits=np.full(n, np.float32(math.log(o / (1 - o)))), sh=np.zeros((n, 16, 3), np.float32))
    out = oracle.render(g, cam_f(W, W, f), W, W)
    o = 1.0 / (1.0 + math.exp(-float(g["opacity_logits"][0])))
    zf = g["means"][:, 2].astype(np.float64)
    s2 = (f / zf) ** 2 + 0.3
    assert np.all(np.ceil(3.0 * np.sqrt(s2 + math.sqrt(0.1))) >= 4)  # every splat covers the image
    jj, ii = np.mgrid[0:W, 0:W].astype(np.float64)
    rho2 = (ii - 4) ** 2 + (jj - 4) ** 2
    total = 0
    for y in range(W):
        for x in range(W):
            T, k = 1.0, 0
            for kk in range(n):
                a = min(0.99, o * math.exp(-0.5 * rho2[y, x] / s2[kk]))
                assert a >= 1.0 / 255.0
                k += 1
                if T * (1.0 - a) < 1e-4:
                    break
                T *= 1.0 - a
            total += k
    assert total < n * W * W  # some pixels stop
    assert out["evals"] == total


def test_contributor_counts_closed_form(oracle):
    # isotropic splats on the axis, alternating faint-and-wide and opaque-and-small:
    # per pixel, n_contrib counts the splats blended (covered, alpha >= 1/255,
    # not stopped) and n_covered the covered splats examined up to and including
    # the last blended one; a faint splat whose square covers a pixel where its
    # alpha is below 1/255 is counted by the second only
    W, f = 21, 10.0
    spec = [(2.0, -1.2, -3.5), (2.4, -2.4, 2.0), (2.8, -1.0, -4.0), (3.2, -2.2, 1.5), (3.6, -1.6, 3.0)]
    z = np.array([s[0] for s in spec], np.float32)
    g = dict(means=np.stack([np.zeros(5), np.zeros(5), z], 1).astype(np.float32),
             log_scales=np.array([[s[1]] * 3 for s in spec], np.float32),
             quats=np.tile(np.float32([1, 0, 0, 0]), (5, 1)),
             opacity_logits=np.array([s[2] for s in spec], np.float32), sh=np.zeros((5, 16, 3), np.float32))
    out = oracle.render(g, cam_f(W, W, f), W, W, mode="pixel")
    c = (W - 1) / 2
    s2 = (f * np.exp(g["log_scales"][:, 0].astype(np.float64)) / z.astype(np.float64)) ** 2 + 0.3
    r = np.ceil(3.0 * np.sqrt(s2 + math.sqrt(0.1)))
    o = 1.0 / (1.0 + np.exp(-g["opacity_logits"].astype(np.float64)))
    n_ref = np.zeros((W, W), np.int32)
    ncov_ref = np.zeros((W, W), np.int32)
    for y in range(W):
        for x in range(W):
            T, n, ncov, last_cov = 1.0, 0, 0, 0
            for k in range(5):
                if max(abs(x - c), abs(y - c)) > r[k]:
                    continue
                ncov += 1
                a = min(0.99, o[k] * math.exp(-0.5 * ((x - c) ** 2 + (y - c) ** 2) / s2[k]))
                if a < 1.0 / 255.0:
                    continue
                if T * (1.0 - a) < 1e-4:
                    break
                T *= 1.0 - a
                n += 1
                last_cov = ncov
            n_ref[y, x], ncov_ref[y, x] = n, last_cov
    assert np.any(ncov_ref > n_ref)  # some covered splat is skipped before a blended one
    np.testing.assert_array_equal(out["n_contrib"], n_ref)
    np.testing.assert_array_equal(out["n_covered"], ncov_ref)


# ---------------------------------------------------------------------------
# camera pose: moving the camera and the scene together changes nothing
# ---------------------------------------------------------------------------
def _grid_scene(n, seed):
    g = synth.box_scene(n, seed=seed)
    g["means"] = (np.round(g["means"] * 1024) / 1024).astype(np.float32)  # exact under the moves below
    g["log_scales"] += np.float32(1.0)
    return g


def test_camera_translation_equivariance(oracle):
    g = _grid_scene(800, 11)
    W, H = 48, 40
    cam0 = cam_f(W, H, 24.0, cx=23.5, cy=19.5)
    C = np.array([3.0, -2.0, 1.5], np.float32)
    cam1 = cam0.copy()
    cam1[9:12] = C
    g1 = dict(g, means=(g["means"] + C).astype(np.float32))
    a = oracle.render(g, cam0, W, H)
    b = oracle.render(g1, cam1, W, H)
    for key in ("rgb", "depth", "T", "n_contrib"):
        assert np.array_equal(a[key], b[key]), key


def test_camera_rotation_equivariance(oracle):
    g = _grid_scene(800, 12)
    g["sh"][:, 1:, :] = 0.0  # view-independent colour
    W, H = 48, 40
    cam0 = cam_f(W, H, 24.0, cx=23.5, cy=19.5)
    P = np.array([[0, 0, -1], [1, 0, 0], [0, -1, 0]], np.float32)  # world->camera rotation
    cam1 = cam0.copy()
    cam1[:9] = P.reshape(9)
    g1 = dict(g, means=(g["means"] @ P).astype(np.float32))  # world points P^T p
    a = oracle.render(g, cam0, W, H)
    g1["quats"] = g["quats"].copy()
    # rotate each Gaussian's frame with the scene: q1 = q(P^T) * q
    qP = Rotation.from_matrix(P.T.astype(np.float64)).as_quat()  # x, y, z, w
    qP = np.array([qP[3], qP[0], qP[1], qP[2]])
    q = g["quats"].astype(np.float64)
    w1, x1, y1, z1 = qP
    w2, x2, y2, z2 = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    g1["quats"] = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    b = oracle.render(g1, cam1, W, H)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-9)
    np.testing.assert_allclose(a["depth"], b["depth"], atol=1e-8)
    assert (a["n_contrib"] != b["n_contrib"]).mean() < 1e-3


# ---------------------------------------------------------------------------
# order: the image depends on the set, not on the input order
# ---------------------------------------------------------------------------
def test_order_independence(oracle):
    n = 1500
    g = synth.box_scene(n, seed=5)
    rng = np.random.default_rng(1)
    g["means"][:, 2] = (2.0 + 4.0 * (rng.permutation(n) + 0.5) / n).astype(np.float32)  # distinct depths
    W = H = 64
    cam = cam_f(W, H, 32.0)
    a = oracle.render(g, cam, W, H)
    perm = rng.permutation(n)
    gp = {k: v[perm] for k, v in g.items()}
    b = oracle.render(gp, cam, W, H)
    for key in ("rgb", "depth", "T", "n_contrib"):
        assert np.array_equal(a[key], b[key]), key


def test_equal_depth_ties_follow_index(oracle):
    # two overlapping splats at the same depth: the lower index is in front
    g = one_gaussian(3.0, -1.5, 2.0, [1.0, 0.0, 0.0])
    h = one_gaussian(3.0, -1.5, 2.0, [0.0, 1.0, 0.0])
    ab = {k: np.concatenate([g[k], h[k]]) for k in g}
    ba = {k: np.concatenate([h[k], g[k]]) for k in g}
    W = H = 9
    cam = cam_f(W, H, 8.0)
    x = oracle.render(ab, cam, W, H)["rgb"][:, 4, 4]
    y = oracle.render(ba, cam, W, H)["rgb"][:, 4, 4]
    assert x[0] > x[1] and y[1] > y[0]


# ---------------------------------------------------------------------------
# loop orders: pixel-major brute force == Gaussian-major walk, bit for bit
# ---------------------------------------------------------------------------
def test_pixel_major_equals_gaussian_major(oracle):
    g = synth.box_scene(2500, seed=0)
    W = H = 128
    cam = synth.identity_camera(W, H)
    a = oracle.render(g, cam, W, H, mode="pixel")
    b = oracle.render(g, cam, W, H, mode="gaussian", nthreads=3)
    for key in ("rgb", "depth", "T", "n_contrib", "amb", "last"):
        assert np.array_equal(a[key], b[key]), key
    assert a["evals"] == b["evals"] > 0


def test_room_view_gaussian_major_matches_pixel_major(oracle):
    g = synth.room_scene(20000, seed=2)
    W, H = 80, 60
    cam = synth.room_camera(2, W, H)
    a = oracle.render(g, cam, W, H, mode="pixel")
    b = oracle.render(g, cam, W, H, mode="gaussian")
    for key in ("rgb", "depth", "T", "n_contrib", "amb"):
        assert np.array_equal(a[key], b[key]), key


# ---------------------------------------------------------------------------
# projection: EWA covariance against the pinhole model
# ---------------------------------------------------------------------------
def _sigma(ls, q):
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return R @ np.diag(np.exp(2 * np.asarray(ls, np.float64))) @ R.T


def _pinhole(p, f, c):
    return np.array([f * p[0] / p[2] + c, f * p[1] / p[2] + c])


def test_ewa_covariance_is_linearised_pinhole(oracle):
    W = H = 64
    f = 32.0
    c = (W - 1) / 2
    rng = np.random.default_rng(7)
    for _ in range(5):
        mu = np.array([rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(2.0, 4.0)], np.float32)
        ls = rng.normal(-3.5, 0.5, 3).astype(np.float32)
        q = rng.standard_normal(4).astype(np.float32)
        g = dict(means=mu[None], log_scales=ls[None], quats=q[None], opacity_logits=np.zeros(1, np.float32),
                 sh=np.zeros((1, 16, 3), np.float32))
        pr = oracle.project(g, cam_f(W, H, f), W, H)
        # Jacobian of the pinhole map by central differences
        p = mu.astype(np.float64)
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            J[:, k] = (_pinhole(p + e, f, c) - _pinhole(p - e, f, c)) / 2e-6
        S2 = J @ _sigma(ls, q) @ J.T
        a, b, cc = pr["cov2"][0]
        np.testing.assert_allclose([a - 0.3, b, cc - 0.3], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-6, atol=1e-9)
        assert pr["u"][0] == pytest.approx(_pinhole(p, f, c)[0], abs=1e-12)
        # conic is the inverse of the dilated covariance; radius from the largest eigenvalue
        M = np.array([[a, b], [b, cc]])
        A, B, C = pr["conic"][0]
        np.testing.assert_allclose(np.array([[A, B], [B, C]]) @ M, np.eye(2), atol=1e-12)
        lam = np.linalg.eigvalsh(M).max()
        if ((a + cc) / 2) ** 2 - (a * cc - b * b) >= 0.1:
            assert pr["radius"][0] == math.ceil(3 * math.sqrt(lam))


def test_ewa_covariance_monte_carlo(oracle):
    # sample the 3D Gaussian, push samples through the pinhole, compare covariances
    W = H = 64
    f = 32.0
    mu = np.array([0.3, -0.2, 3.0], np.float32)
    ls = np.log(np.array([0.02, 0.05, 0.01], np.float32))
    q = np.array([0.9, 0.2, -0.3, 0.25], np.float32)
    g = dict(means=mu[None], log_scales=ls[None], quats=q[None], opacity_logits=np.zeros(1, np.float32),
             sh=np.zeros((1, 16, 3), np.float32))
    pr = oracle.project(g, cam_f(W, H, f), W, H)
    rng = np.random.default_rng(0)
    x = rng.multivariate_normal(mu.astype(np.float64), _sigma(ls, q), size=400_000)
    uv = np.stack([f * x[:, 0] / x[:, 2], f * x[:, 1] / x[:, 2]], 1)
    Cmc = np.cov(uv.T)
    a, b, c = pr["cov2"][0]
    scale = max(a, c)
    assert abs(a - 0.3 - Cmc[0, 0]) < 1e-2 * scale
    assert abs(c - 0.3 - Cmc[1, 1]) < 1e-2 * scale
    assert abs(b - Cmc[0, 1]) < 1e-2 * scale


def test_lateral_clamp_of_jacobian(oracle):
    # beyond 1.3 x the half field the Jacobian's x/z is held at the limit
    W = H = 64
    f = 32.0
    mu = np.array([4.0, 0.0, 1.0], np.float32)  # x/z = 4 > 1.3
    g = dict(means=mu[None], log_scales=np.full((1, 3), -2.0, np.float32), quats=np.float32([[1, 0, 0, 0]]),
             opacity_logits=np.zeros(1, np.float32), sh=np.zeros((1, 16, 3), np.float32))
    pr = oracle.project(g, cam_f(W, H, f), W, H)
    s2 = math.exp(2 * float(np.float32(-2.0)))
    lim = 1.3 * (W / 2) / f
    J = np.array([[f / 1.0, 0.0, -f * lim / 1.0], [0.0, f / 1.0, 0.0]])
    S2 = J @ (s2 * np.eye(3)) @ J.T
    np.testing.assert_allclose(pr["cov2"][0], [S2[0, 0] + 0.3, S2[0, 1], S2[1, 1] + 0.3], rtol=1e-12)


def test_near_plane_cull_uses_fp32_key(oracle):
    W = H = 16
    zs = [0.1, 0.2, np.nextafter(np.float32(0.2), np.float32(1)), 0.5]
    g = dict(means=np.array([[0, 0, z] for z in zs], np.float32), log_scales=np.full((4, 3), -3.0, np.float32),
             quats=np.tile(np.float32([1, 0, 0, 0]), (4, 1)), opacity_logits=np.zeros(4, np.float32),
             sh=np.zeros((4, 16, 3), np.float32))
    pr = oracle.project(g, cam_f(W, H, 8.0), W, H)
    assert pr["visible"].tolist() == [False, False, True, True]


# ---------------------------------------------------------------------------
# rotation and spherical harmonics against library routines
# ---------------------------------------------------------------------------
def test_quaternion_rotation(oracle):
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.standard_normal(4)
        R = oracle.quat_to_rot(q)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_array_equal(R, oracle.quat_to_rot(-q))
        qn = q / np.linalg.norm(q)
        Rs = Rotation.from_quat([qn[1], qn[2], qn[3], qn[0]]).as_matrix()
        np.testing.assert_allclose(R, Rs, atol=1e-14)


def test_sh_orthonormal_by_quadrature(oracle):
    x, w = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wt = (w[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).reshape(-1)
    Y = oracle.sh_basis(d)
    gram = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)
    assert Y[0, 0] == pytest.approx(0.28209479177387814, abs=1e-16)


def test_sh_matches_scipy_real_harmonics(oracle):
    sp = pytest.importorskip("scipy.special")
    f = getattr(sp, "sph_harm_y", None)
    rng = np.random.default_rng(0)
    d = rng.standard_normal((64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    th, ph = np.arccos(d[:, 2]), np.arctan2(d[:, 1], d[:, 0])
    if f is None:  # older scipy: sph_harm(m, l, azimuth, polar)
        f = lambda l, m, t, p: sp.sph_harm(m, l, p, t)  # noqa: E731
    Y = oracle.sh_basis(d)
    for l in range(4):
        for m in range(-l, l + 1):
            if m > 0:
                std = math.sqrt(2) * (-1) ** m * f(l, m, th, ph).real
            elif m < 0:
                std = math.sqrt(2) * (-1) ** m * f(l, -m, th, ph).imag
            else:
                std = f(l, 0, th, ph).real
            # 3DGS ordering index l^2 + l + m; odd-m functions carry a minus sign
            np.testing.assert_allclose(Y[:, l * l + l + m], (-1) ** m * std, atol=1e-13)


def test_colour_clamped_at_zero_and_direction_dependent(oracle):
    W = H = 9
    g = one_gaussian(3.0, -2.0, 2.0, [-2.0, 0.0, 0.0], xy=(0.5, 0.0))
    g["sh"][0, 3, :] = 0.5  # Y_{1,1} = -c1 x term
    pr = oracle.project(g, cam_f(W, H, 8.0), W, H)
    d = np.array([0.5, 0.0, 3.0]) / np.linalg.norm([0.5, 0.0, 3.0])
    c1 = math.sqrt(3 / (4 * math.pi))
    raw = C0 * np.float32([-2.0, 0.0, 0.0]) + 0.5 + (-c1 * d[0]) * 0.5
    np.testing.assert_allclose(pr["rgb"][0], np.maximum(raw, 0.0), atol=1e-14)
    assert pr["rgb"][0][0] == 0.0


# ---------------------------------------------------------------------------
# linear blend skinning
# ---------------------------------------------------------------------------
def _avatar(n=64, seed=0):
    a = synth.avatar_canonical(n, seed)
    return a


def test_lbs_identity(oracle):
    a = _avatar()
    n = a["means"].shape[0]
    G = np.zeros((1, 24, 3, 4))
    G[:, :, :, :3] = np.eye(3)
    w = a["weights"].astype(np.float64)
    w /= w.sum(1, keepdims=True)
    m, c = oracle.lbs(a["means"], a["log_scales"], a["quats"], a["joint_ids"], w, np.zeros(n, np.int32), G)
    np.testing.assert_allclose(m, a["means"].astype(np.float64), atol=1e-15)
    for i in range(n):
        S = _sigma(a["log_scales"][i], a["quats"][i])
        np.testing.assert_allclose(c[i], [S[0, 0], S[0, 1], S[0, 2], S[1, 1], S[1, 2], S[2, 2]], rtol=1e-12, atol=1e-18)


def test_lbs_common_rigid_transform_and_no_renormalisation(oracle):
    a = _avatar(seed=1)
    n = a["means"].shape[0]
    Q = Rotation.from_rotvec([0.3, -0.5, 0.8]).as_matrix()
    t = np.array([1.0, 2.0, 0.9])
    G = np.zeros((2, 24, 3, 4))
    G[:, :, :, :3] = Q
    G[:, :, :, 3] = t
    w = a["weights"].astype(np.float64) * 0.9  # weights used as given
    av = np.arange(n, dtype=np.int32) % 2
    m, c = oracle.lbs(a["means"], a["log_scales"], a["quats"], a["joint_ids"], w, av, G)
    sw = w.sum(1)
    np.testing.assert_allclose(m, sw[:, None] * (a["means"].astype(np.float64) @ Q.T + t), atol=1e-13)
    for i in range(0, n, 7):
        S = _sigma(a["log_scales"][i], a["quats"][i])
        P = sw[i] ** 2 * Q @ S @ Q.T
        np.testing.assert_allclose(c[i], [P[0, 0], P[0, 1], P[0, 2], P[1, 1], P[1, 2], P[2, 2]], rtol=1e-11, atol=1e-18)


def test_zero_pose_forward_kinematics_is_identity():
    M = synth.forward_kinematics(np.zeros((24, 3)), [0.0, 0.0, 0.0])
    I = np.zeros((24, 3, 4))
    I[:, :, :3] = np.eye(3)
    np.testing.assert_allclose(M, I, atol=1e-15)
    # a pure root translation moves every joint's skinning matrix by it
    M = synth.forward_kinematics(np.zeros((24, 3)), [1.0, 2.0, 3.0])
    np.testing.assert_allclose(M[:, :, 3], np.tile([1.0, 2.0, 3.0], (24, 1)), atol=1e-15)
