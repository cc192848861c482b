"""Pins of the oracle's avatar-driving and composite functions (CPU only):
forward kinematics of the joint tree and the interpolation of per-frame joint
matrices (Sec. 3.3.1), and the nearest-fragment composite of two layers
(Sec. 3.2).  Each is pinned to facts outside its own code: rigid-body
invariants, closed forms and the oracle renderer."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2604_12626_gb300 import synth

J = synth.N_JOINTS


def _pose(seed, A=3, sigma=0.4):
    rng = np.random.default_rng(seed)
    local = Rotation.from_rotvec(rng.normal(0, sigma, (A * J, 3))).as_matrix().reshape(A, J, 3, 3)
    root = np.zeros((A, 3, 4))
    root[:, :, :3] = Rotation.from_rotvec(rng.normal(0, 1.0, (A, 3))).as_matrix()
    root[:, :, 3] = rng.uniform(-3, 3, (A, 3))
    return local, root


def _posed_joints(M, rest):
    """Posed joint positions M_j [J_j; 1] (the translation of G_j)."""
    return np.einsum("ajrc,jc->ajr", M[..., :3], rest) + M[..., 3]


def test_fk_zero_pose_is_identity(oracle):
    local = np.tile(np.eye(3), (2, J, 1, 1))
    root = np.zeros((2, 3, 4))
    root[:, :, :3] = np.eye(3)
    M = oracle.forward_kinematics(local, root, synth.REST_JOINTS, synth.PARENTS)
    assert synth.REST_JOINTS[0].tolist() == [0.0, 0.0, 0.0]
    np.testing.assert_allclose(M, np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]), (2, J, 1, 1)), atol=1e-15)


def test_fk_rigid_invariants(oracle):
    local, root = _pose(1)
    M = oracle.forward_kinematics(local, root, synth.REST_JOINTS, synth.PARENTS)
    R = M[..., :3]
    # every global rotation is orthonormal with determinant 1
    np.testing.assert_allclose(np.einsum("ajrc,ajsc->ajrs", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
    # bone lengths are preserved by any pose
    p = _posed_joints(M, synth.REST_JOINTS)
    for j in range(1, J):
        q = synth.PARENTS[j]
        np.testing.assert_allclose(np.linalg.norm(p[:, j] - p[:, q], axis=-1),
                                   np.linalg.norm(synth.REST_JOINTS[j] - synth.REST_JOINTS[q]), atol=1e-12)
    # the root joint sits at the root translation
    np.testing.assert_allclose(p[:, 0], root[:, :, 3], atol=1e-12)


def test_fk_rotating_one_joint_moves_only_its_subtree(oracle):
    local, root = _pose(2, A=1)
    k = 9  # a spine joint with arms and head below it
    local2 = local.copy()
    local2[0, k] = Rotation.from_rotvec([0.3, -0.2, 0.5]).as_matrix() @ local2[0, k]
    M1 = oracle.forward_kinematics(local, root, synth.REST_JOINTS, synth.PARENTS)
    M2 = oracle.forward_kinematics(local2, root, synth.REST_JOINTS, synth.PARENTS)
    desc = {k}
    for j in range(J):
        if synth.PARENTS[j] in desc:
            desc.add(j)
    moved = [j for j in range(J) if not np.allclose(M1[0, j], M2[0, j], atol=1e-14)]
    assert set(moved) == desc
    # joint k's own position does not move (it rotates about itself)
    p1, p2 = _posed_joints(M1, synth.REST_JOINTS), _posed_joints(M2, synth.REST_JOINTS)
    np.testing.assert_allclose(p1[0, k], p2[0, k], atol=1e-12)


def test_fk_root_equivariance(oracle):
    local, root = _pose(3)
    Q = Rotation.from_rotvec([0.2, 0.9, -0.4]).as_matrix()
    b = np.array([1.0, -2.0, 0.5])
    root2 = root.copy()
    root2[:, :, :3] = Q @ root[:, :, :3]
    root2[:, :, 3] = root[:, :, 3] @ Q.T + b
    M1 = oracle.forward_kinematics(local, root, synth.REST_JOINTS, synth.PARENTS)
    M2 = oracle.forward_kinematics(local, root2, synth.REST_JOINTS, synth.PARENTS)
    np.testing.assert_allclose(M2[..., :3], Q @ M1[..., :3], atol=1e-12)
    np.testing.assert_allclose(M2[..., 3], M1[..., 3] @ Q.T + b, atol=1e-12)


def test_fk_matches_the_synthetic_pose_generator(oracle):
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 0.3, (J, 3))
    yaw, t = 1.1, np.array([2.0, 3.0, 0.9])
    local = Rotation.from_rotvec(theta).as_matrix()[None]
    root = np.zeros((1, 3, 4))
    root[0, :, :3] = Rotation.from_rotvec([0, 0, yaw]).as_matrix()
    root[0, :, 3] = t
    M = oracle.forward_kinematics(local, root, synth.REST_JOINTS, synth.PARENTS)[0]
    np.testing.assert_allclose(M, synth.forward_kinematics(theta, t, yaw), atol=1e-12)


def test_interpolation_between_frames(oracle):
    rng = np.random.default_rng(5)
    A, F = 2, 5
    frames = rng.normal(size=(A, F, J, 3, 4))
    for f in range(F):
        np.testing.assert_array_equal(oracle.interpolate_frames(frames, [f, f]), frames[:, f])
    mid = oracle.interpolate_frames(frames, [1.5, 2.25])
    np.testing.assert_allclose(mid[0], 0.5 * (frames[0, 1] + frames[0, 2]), atol=1e-15)
    np.testing.assert_allclose(mid[1], 0.75 * frames[1, 2] + 0.25 * frames[1, 3], atol=1e-15)
    # clamped outside the clip
    np.testing.assert_array_equal(oracle.interpolate_frames(frames, [-3.0, 99.0])[0], frames[0, 0])
    np.testing.assert_array_equal(oracle.interpolate_frames(frames, [-3.0, 99.0])[1], frames[1, F - 1])
    # a pose held over all frames stays that pose
    held = np.repeat(frames[:, :1], F, axis=1)
    np.testing.assert_allclose(oracle.interpolate_frames(held, [0.3, 3.7]), frames[:, 0], atol=1e-15)


def test_composite_picks_the_nearer_fragment(oracle):
    # hand-made pixels: (D_a, D_b) and which layer the composite keeps
    cases = [(1.0, 2.0, "a"), (2.0, 1.0, "b"), (1.5, 1.5, "b"), (0.0, 2.0, "b"), (1.0, 0.0, "a"), (0.0, 0.0, "b"),
             (math.inf, 3.0, "b"), (math.nan, 3.0, "b"), (2.0, -1.0, "a")]
    n = len(cases)
    da = np.array([[[c[0] for c in cases]]])
    db = np.array([[[c[1] for c in cases]]])
    ra = np.broadcast_to(np.array([0.1, 0.2, 0.3])[None, :, None, None], (1, 3, 1, n)).copy()
    rb = np.broadcast_to(np.array([0.7, 0.8, 0.9])[None, :, None, None], (1, 3, 1, n)).copy()
    rgb, dep = oracle.composite_nearest(ra, da, rb, db)
    for i, (_, _, w) in enumerate(cases):
        src_rgb, src_d = (ra, da) if w == "a" else (rb, db)
        np.testing.assert_array_equal(rgb[0, :, 0, i], src_rgb[0, :, 0, i])
        assert dep[0, 0, i] == src_d[0, 0, i] or (np.isnan(dep[0, 0, i]) and np.isnan(src_d[0, 0, i]))


def test_composite_of_two_renders_matches_the_joint_render_where_opaque(oracle):
    """A far layer and a near opaque one rendered separately and composited by
    normalised depth equal the joint render wherever the near layer alone
    decides the pixel (the joint render blends nothing of the far layer there:
    same final transmittance), and show the far layer where the near one is
    absent."""
    rng = np.random.default_rng(6)

    def layer(n, z, spread):
        return dict(means=np.stack([rng.uniform(-spread, spread, n), rng.uniform(-spread, spread, n),
                                    rng.uniform(z, z + 0.05, n)], 1).astype(np.float32),
                    log_scales=np.full((n, 3), -2.0, np.float32), quats=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
                    opacity_logits=np.full(n, 6.0, np.float32),
                    sh=rng.normal(0, 0.3, (n, 16, 3)).astype(np.float32))

    far, near = layer(600, 4.0, 1.6), layer(150, 2.0, 0.35)
    joint = {k: np.concatenate([far[k], near[k]]) for k in far}
    W = H = 32
    cam = synth.identity_camera(W, H)
    rf = oracle.render(far, cam, W, H, normalize_depth=True)
    rn = oracle.render(near, cam, W, H, normalize_depth=True)
    rj = oracle.render(joint, cam, W, H, normalize_depth=True)
    rgb, dep = oracle.composite_nearest(rn["rgb"][None], rn["depth"][None], rf["rgb"][None], rf["depth"][None])
    opaque_near = (rj["T"] == rn["T"]) & (rn["T"] < 1e-2)
    assert opaque_near.sum() > 50 and (~opaque_near).sum() > 50
    np.testing.assert_allclose(rgb[0][:, opaque_near], rj["rgb"][:, opaque_near], atol=1e-5)
    np.testing.assert_allclose(dep[0][opaque_near], rj["depth"][opaque_near], rtol=1e-5)
    # where the near layer is absent the far layer shows through unchanged
    absent = rn["T"] == 1.0
    np.testing.assert_array_equal(rgb[0][:, absent], rf["rgb"][:, absent])


def test_sh_direction_matrix(oracle):
    """Colour of a posed avatar Gaussian evaluated in its canonical frame: the
    SH direction is M (mu - C) normalised.  Identity (or any positive scaling)
    changes nothing; a rotation gives the closed-form degree-1 colour."""
    rng = np.random.default_rng(9)
    n = 200
    g = synth.box_scene(n, seed=9)
    cam = synth.identity_camera(64, 64)
    base = oracle.render(g, cam, 64, 64)
    r = oracle.render(dict(g, sh_dirmat=np.tile(np.eye(3).reshape(1, 9), (n, 1))), cam, 64, 64)
    for k in ("rgb", "depth", "T", "n_contrib"):
        np.testing.assert_array_equal(r[k], base[k])
    r = oracle.render(dict(g, sh_dirmat=np.tile(2.5 * np.eye(3).reshape(1, 9), (n, 1))), cam, 64, 64)
    np.testing.assert_allclose(r["rgb"], base["rgb"], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(r["n_contrib"], base["n_contrib"])
    # one Gaussian on the optical axis: direction (0, 0, 1), rotated by M
    k0 = np.array([0.3, -0.1, 0.2])
    k1 = rng.normal(0, 0.3, (3, 3))  # rows: the three degree-1 functions, columns: channels
    sh = np.zeros((1, 16, 3))
    sh[0, 0], sh[0, 1:4] = k0, k1
    one = dict(means=np.array([[0.0, 0.0, 3.0]]), log_scales=np.full((1, 3), -2.0), quats=np.array([[1.0, 0, 0, 0]]),
               opacity_logits=np.zeros(1), sh=sh)
    M = Rotation.from_rotvec([0.4, -0.7, 0.2]).as_matrix()
    x, y, z = M @ np.array([0.0, 0.0, 1.0])
    c0, c1 = 0.5 / math.sqrt(math.pi), math.sqrt(3.0 / (4.0 * math.pi))
    expect = np.maximum(0.0, 0.5 + c0 * k0 + c1 * (-y * k1[0] + z * k1[1] - x * k1[2]))
    p = oracle.project(dict(one, sh_dirmat=M.reshape(1, 9)), cam, 64, 64)
    np.testing.assert_allclose(p["rgb"][0], expect, atol=1e-14)


# ---------------------------------------------------------------------------
# triangle-mesh layer (the mesh pass of the composite, Sec. 3.2)
# ---------------------------------------------------------------------------
def _ray(i, j, f, c):
    return np.stack([(i - c) / f, (j - c) / f, np.ones_like(i)], -1)


def test_mesh_depth_is_the_ray_plane_intersection_and_colour_the_surface_point(oracle):
    W, f = 48, 30.0
    c = (W - 1) / 2
    cam = synth.identity_camera(W, W)
    cam[12:16] = [f, f, c, c]
    P = np.array([[-1.2, -0.9, 3.0], [1.4, -0.5, 4.5], [-0.2, 1.3, 2.2]])
    m = oracle.raster_mesh(P, P * 0.1, [[0, 1, 2]], cam, W, W)  # colour = 0.1 x the vertex position
    jj, ii = np.mgrid[0:W, 0:W].astype(np.float64)
    r = _ray(ii, jj, f, c)
    n = np.cross(P[1] - P[0], P[2] - P[0])
    t = (n @ P[0]) / (r @ n)
    cov = (m["depth"] > 0) & (m["amb"] == 0)
    assert cov.sum() > 200
    np.testing.assert_allclose(m["depth"][cov], t[cov], rtol=1e-12)
    surf = r * t[..., None] * 0.1
    np.testing.assert_allclose(np.moveaxis(m["rgb"], 0, -1)[cov], surf[cov], rtol=1e-11, atol=1e-13)


def test_mesh_coverage_of_a_right_triangle(oracle):
    W, f = 40, 20.0
    c = (W - 1) / 2
    cam = synth.identity_camera(W, W)
    cam[12:16] = [f, f, c, c]
    z, x0, y0, L = 2.0, 5.5, 7.5, 20.0  # screen vertices (x0, y0), (x0 + L, y0), (x0, y0 + L)
    scr = np.array([[x0, y0], [x0 + L, y0], [x0, y0 + L]])
    P = np.concatenate([(scr - c) / f * z, np.full((3, 1), z)], 1)
    m = oracle.raster_mesh(P, np.ones((3, 3)), [[0, 1, 2]], cam, W, W, bg=(0.2, 0.2, 0.2))
    jj, ii = np.mgrid[0:W, 0:W]
    want = (ii >= x0) & (jj >= y0) & ((ii - x0) + (jj - y0) <= L)
    ok = m["amb"] == 0
    np.testing.assert_array_equal((m["depth"] > 0)[ok], want[ok])
    np.testing.assert_allclose(m["depth"][want & ok], z, rtol=1e-14)
    np.testing.assert_allclose(m["rgb"][:, ~want], 0.2)
    assert np.all(((ii - x0) + (jj - y0))[~ok] == L)  # only centres on the hypotenuse's line are flagged


def test_mesh_occlusion_ties_and_near_cull(oracle):
    W, f = 32, 16.0
    c = (W - 1) / 2
    cam = synth.identity_camera(W, W)
    cam[12:16] = [f, f, c, c]
    quad = lambda z, s: np.array([[-s, -s, z], [s, -s, z], [s, s, z], [-s, s, z]])  # noqa: E731
    V = np.concatenate([quad(3.0, 2.0), quad(2.0, 0.8), quad(2.0, 0.8), [[0, 0, 0.1], [1, 0, 3], [0, 1, 3]]])
    col = np.concatenate([np.full((4, 3), 0.1), np.full((4, 3), 0.5), np.full((4, 3), 0.9), np.full((3, 3), 0.7)])
    T = [[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7], [8, 9, 10], [8, 10, 11], [12, 13, 14]]
    m = oracle.raster_mesh(V, col, T, cam, W, W)
    ok = m["amb"] == 0
    front = (np.abs(np.mgrid[0:W, 0:W][1] - c) < 0.8 / 2.0 * f - 0.5) & (np.abs(np.mgrid[0:W, 0:W][0] - c) < 0.8 / 2.0 * f - 0.5)
    assert front.sum() > 20
    # (inside the near quad, away from its edges: the exact tie between the two
    # copies is flagged for FP32, but the definition decides it by index)
    np.testing.assert_allclose(m["depth"][front], 2.0)  # the near quad hides the far one
    np.testing.assert_allclose(m["rgb"][:, front], 0.5)  # equal depths: the lower triangle index wins
    back = (m["depth"] > 2.5) & ok
    assert back.sum() > 100
    np.testing.assert_allclose(m["rgb"][:, back], 0.1)
    assert not np.any(np.isclose(m["rgb"][0], 0.7))  # the triangle through the near plane is culled
