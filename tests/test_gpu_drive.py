"""Avatar driving and the sensor composite on the GPU against the FP64 oracle:
forward kinematics and keyframe interpolation of the joint matrices
(Sec. 3.3.1), and the nearest-fragment composite of two RGB-D layers
(Sec. 3.2), alone and chained with LBS and the renderer."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import compare_view  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402
from test_gpu_deform import gpu_avatars, make_avatars  # noqa: E402

J = synth.N_JOINTS


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def T(x, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)


def random_pose(seed, A, sigma=0.3):
    rng = np.random.default_rng(seed)
    local = Rotation.from_rotvec(rng.normal(0, sigma, (A * J, 3))).as_matrix().reshape(A, J, 3, 3)
    root = np.zeros((A, 3, 4))
    root[:, :, :3] = Rotation.from_rotvec(np.stack([np.zeros(A), np.zeros(A), rng.uniform(0, 6.28, A)], 1)).as_matrix()
    root[:, :, 3] = np.stack([rng.uniform(0.5, 9.5, A), rng.uniform(0.5, 7.5, A), np.full(A, 0.9)], 1)
    return local.astype(np.float32), root.astype(np.float32)


@pytest.mark.parametrize("A", [1, 37, 256])
def test_forward_kinematics_matches_oracle(gs, oracle, A):
    local, root = random_pose(A, A)
    rest = synth.REST_JOINTS.astype(np.float32)
    M = gs.forward_kinematics(T(local), T(root), T(rest), synth.PARENTS)
    torch.cuda.synchronize()
    ref = oracle.forward_kinematics(local, root, rest, synth.PARENTS)
    np.testing.assert_allclose(M.cpu().numpy(), ref, rtol=0, atol=2e-5)


def test_forward_kinematics_rejects_a_parent_below_its_child(gs):
    local, root = random_pose(0, 2)
    bad = synth.PARENTS.copy()
    bad[5] = 7
    with pytest.raises(gs.GsError, match="INVALID_ARG"):
        gs.forward_kinematics(T(local), T(root), T(synth.REST_JOINTS.astype(np.float32)), bad)


def test_interpolate_joints_matches_oracle(gs, oracle):
    A, F = 16, 30
    rng = np.random.default_rng(3)
    frames = np.stack([np.stack([synth.random_pose(100 * a + f) for f in range(F)]) for a in range(A)])
    t = np.concatenate([rng.uniform(0, F - 1, A - 4), [0.0, F - 1.0, -2.5, F + 4.0]]).astype(np.float32)
    out = gs.interpolate_joints(T(frames), T(t))
    torch.cuda.synchronize()
    ref = oracle.interpolate_frames(frames, t)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-6 * (np.abs(frames).max() + 1))
    # whole frames come back bit for bit
    np.testing.assert_array_equal(out[A - 4].cpu().numpy(), frames[A - 4, 0])
    np.testing.assert_array_equal(out[A - 3].cpu().numpy(), frames[A - 3, F - 1])


@pytest.mark.parametrize("H,W", [(64, 64), (37, 29)])  # float4 path and scalar path
def test_composite_matches_oracle_bit_exact(gs, oracle, H, W):
    V = 3
    rng = np.random.default_rng(H)
    da = rng.uniform(0.5, 5.0, (V, H, W)).astype(np.float32)
    db = rng.uniform(0.5, 5.0, (V, H, W)).astype(np.float32)
    # uncovered pixels, ties and non-finite depths
    da[:, ::7] = 0.0
    db[:, :, ::5] = 0.0
    db[:, 3, :] = da[:, 3, :]
    da[0, 1, :4] = np.inf
    db[1, 2, :4] = np.nan
    da[2, 4, :4] = -1.0
    ra = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    rb = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    rgb, dep = gs.composite_nearest(T(ra), T(da), T(rb), T(db))
    torch.cuda.synchronize()
    ref_rgb, ref_dep = oracle.composite_nearest(ra, da, rb, db)
    np.testing.assert_array_equal(rgb.cpu().numpy(), ref_rgb.astype(np.float32))
    np.testing.assert_array_equal(dep.cpu().numpy(), ref_dep.astype(np.float32))
    # in place on the first layer
    A_rgb, A_dep = T(ra), T(da)
    gs.composite_nearest(A_rgb, A_dep, T(rb), T(db), out=(A_rgb, A_dep))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(A_rgb.cpu().numpy(), ref_rgb.astype(np.float32))


def test_drive_deform_and_composite_chain(gs, oracle):
    """Keyframes interpolated at the simulation time, LBS, the scene and the
    avatars rendered as two layers with normalised depth, then composited --
    the two-pass sensor of Sec. 3.2 on one stream -- against the same chain on
    the oracle.  Each layer is compared with the renderer's tolerances and the
    composite of the GPU layers must be the oracle's selection bit for bit."""
    W = H = 96
    n_room, n_av, n_avatars, F = 80_000, 4000, 2, 8
    room = synth.room_scene(n_room, seed=500)
    cam = synth.room_camera(500, W, H)
    av, _, avatar_of = make_avatars(n_avatars, n_av, 50)
    fwd, C = cam[6:9], cam[9:12]
    frames = np.stack([np.stack([synth.random_pose(10 * a + f) for f in range(F)]) for a in range(n_avatars)])
    for a in range(n_avatars):  # every keyframe 2-2.5 m in front of the camera
        root = C + fwd * (2.0 + 0.5 * a) + np.array([0.0, 0.0, -0.3])
        frames[a, :, :, :, 3] += (root - frames[a, :, 0, :, 3])[:, None, :].astype(np.float32)
    t = np.array([2.25, 5.5], np.float32)
    G = gs.interpolate_joints(T(frames), T(t))
    m = n_av * n_avatars
    A = gpu_avatars(gs, av, avatar_of, n_avatars)
    av_g = gs.Gaussians.from_numpy({k: av[k] for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
                                   | {"cov3d": np.zeros((m, 6), np.float32)})
    gs.deform(A, G, av_g.means, av_g.cov3d)
    kw = dict(normalize_depth=True)
    r_scene = gs.Renderer(gs.Batch(np.array([0, n_room])), W, H, **kw)
    r_av = gs.Renderer(gs.Batch(np.array([0, m]), env_cov3d_begin=[0]), W, H, **kw)
    ct = gs.cameras_tensor(cam[None])
    out_s = r_scene.forward(gs.Gaussians.from_numpy(room), ct)
    out_a = r_av.forward(av_g, ct)
    rgb, dep = gs.composite_nearest(out_a[0], out_a[1], out_s[0], out_s[1])
    torch.cuda.synchronize()
    # the oracle chain
    Gref = oracle.interpolate_frames(frames, t)
    pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32), av["weights"],
                        avatar_of, Gref)
    ge = {k: av[k].astype(np.float64) for k in ("log_scales", "quats", "opacity_logits", "sh")}
    ge.update(means=pm, cov3d=pc, use_cov=np.ones(m, np.uint8), inexact=np.ones(m, np.uint8))
    ora_a = oracle.render(ge, cam, W, H, normalize_depth=True)
    ora_s = oracle.render(room, cam, W, H, normalize_depth=True)
    for out, ora in ((out_a, ora_a), (out_s, ora_s)):
        compare_view(dict(rgb=out[0][0].cpu().numpy(), depth=out[1][0].cpu().numpy(), T=out[2][0].cpu().numpy(),
                          n_contrib=out[3][0].cpu().numpy()), ora)
    assert (ora_a["T"] < 0.5).mean() > 0.02  # the avatars are in view
    sel_rgb, sel_dep = oracle.composite_nearest(out_a[0].cpu().numpy(), out_a[1].cpu().numpy(),
                                                out_s[0].cpu().numpy(), out_s[1].cpu().numpy())
    np.testing.assert_array_equal(rgb.cpu().numpy(), sel_rgb.astype(np.float32))
    np.testing.assert_array_equal(dep.cpu().numpy(), sel_dep.astype(np.float32))


def test_exp2_rate_kernel(gs):
    """The exp2 throughput kernel computes what it claims: eight chains of
    x <- 2^(-x) per thread, which converge to the fixed point 0.6412 (the
    contraction factor is ln 2 * 2^(-x) < 0.5)."""
    out = torch.empty(2 * 256, device="cuda")
    n = gs.exp2_rate(2, 32, out)
    torch.cuda.synchronize()
    assert n == 2 * 256 * 32 * 8
    np.testing.assert_allclose(out.cpu().numpy() / 8.0, 0.641185744, atol=1e-4)
    with pytest.raises(gs.GsError, match="INVALID_ARG"):
        gs.exp2_rate(0, 32, out)


def _capsule_scene(gs, oracle, seed, avatars_per_env=(3, 0, 8, 1)):
    """Capsules of avatars posed by FK in several rooms (envs), from the CUDA
    path and from the oracle, with their env offsets."""
    A = sum(avatars_per_env)
    local, root = random_pose(seed, A)
    rest = synth.REST_JOINTS.astype(np.float32)
    radius = np.linspace(0.06, 0.12, J).astype(np.float32)
    M = gs.forward_kinematics(T(local), T(root), T(rest), synth.PARENTS)
    caps = gs.avatar_capsules(M, T(rest), synth.PARENTS, T(radius))
    torch.cuda.synchronize()
    ref = oracle.avatar_capsules(M.cpu().numpy(), rest, synth.PARENTS, radius)
    off = np.concatenate([[0], np.cumsum(np.asarray(avatars_per_env) * J)]).astype(np.int64)
    return caps, ref, off


def test_avatar_capsules_match_oracle(gs, oracle):
    caps, ref, _ = _capsule_scene(gs, oracle, 5)
    np.testing.assert_allclose(caps.cpu().numpy(), ref, rtol=0, atol=2e-6)
    assert np.all(caps.cpu().numpy()[:, 0, :3] == caps.cpu().numpy()[:, 0, 4:7])  # the root: a sphere


@pytest.mark.parametrize("with_step", [False, True])
def test_capsule_queries_match_oracle(gs, oracle, with_step):
    """Per query: distance and nearest capsule, and for a step the blocked flag
    and the first-contact fraction, against the FP64 oracle on the same
    capsules.  A query whose answer an FP32 rounding could change (a second
    capsule within 1e-5 m of the nearest, or contact within 1e-4 m of grazing:
    the oracle's flag differs at agent radius r -/+ 1e-4) is left out of the
    comparison of that answer; there are few of them."""
    caps, _, off = _capsule_scene(gs, oracle, 9)
    capf = caps.reshape(-1, 8)
    capn = capf.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(11)
    Q, r = 4000, 0.1
    qe = rng.integers(0, len(off) - 1, Q).astype(np.int32)
    p0 = np.stack([rng.uniform(0.0, 10.0, Q), rng.uniform(0.0, 8.0, Q), rng.uniform(0.1, 1.8, Q)], 1)
    step = rng.normal(0.0, 0.4, (Q, 3))
    step[:, 2] *= 0.1
    p1 = p0 + step
    # queries near the avatars, so that contacts and small distances occur
    ci = rng.integers(0, capn.shape[0], Q)
    near = rng.uniform(0, 1, Q) < 0.5
    base = capn[ci, :3] + rng.normal(0, 0.3, (Q, 3))
    envs_of_cap = np.searchsorted(off, ci, side="right") - 1
    p0[near] = base[near]
    qe[near] = envs_of_cap[near]
    p1[near] = p0[near] + step[near]
    p0 = p0.astype(np.float32)
    p1 = p1.astype(np.float32)
    d_off = torch.from_numpy(off).cuda()
    dist, nearest, tclip, blocked = gs.capsule_query(capf, d_off, T(qe, torch.int32), T(p0),
                                                     T(p1) if with_step else None, agent_radius=r)
    torch.cuda.synchronize()
    ref = oracle.capsule_query(capn, off, qe, p0, p1 if with_step else None, agent_radius=r)
    dist, nearest, tclip, blocked = (x.cpu().numpy() for x in (dist, nearest, tclip, blocked))
    has = off[qe + 1] > off[qe]
    assert np.all(np.isinf(dist[~has])) and np.all(nearest[~has] == -1) and not blocked[~has].any()
    np.testing.assert_allclose(dist[has], ref["dist"][has], rtol=0, atol=2e-5)
    # nearest capsule, except where a second one is within 1e-5 m
    second = np.full(Q, np.inf)
    for q in np.flatnonzero(has):
        c = capn[off[qe[q]]:off[qe[q] + 1]]
        ab = c[:, 4:7] - c[:, :3]
        s = np.clip(((p0[q] - c[:, :3]) * ab).sum(1) / np.maximum((ab * ab).sum(1), 1e-300), 0.0, 1.0)
        d = np.linalg.norm(p0[q] - (c[:, :3] + s[:, None] * ab), axis=1) - c[:, 3]
        second[q] = np.sort(d)[1] - np.sort(d)[0] if d.size > 1 else np.inf
    clear = has & (second > 1e-5)
    assert np.array_equal(nearest[clear], ref["nearest"][clear])
    assert clear.mean() > 0.5
    lo = oracle.capsule_query(capn, off, qe, p0, p1 if with_step else None, agent_radius=r - 1e-4)["blocked"]
    hi = oracle.capsule_query(capn, off, qe, p0, p1 if with_step else None, agent_radius=r + 1e-4)["blocked"]
    firm = lo == hi
    assert firm.mean() > 0.99
    assert np.array_equal(blocked.astype(bool)[firm], ref["blocked"][firm])
    if with_step:
        both = firm & ref["blocked"]
        assert both.sum() > 100  # contacts are exercised
        np.testing.assert_allclose(tclip[both], ref["tclip"][both], rtol=0, atol=2e-3)
        assert np.all(tclip[firm & ~ref["blocked"]] == 1.0)
