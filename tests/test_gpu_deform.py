"""LBS deformation on the GPU (gs_deform_avatars and its adjoint) against the
FP64 oracle, and scenes with avatars rendered in one pass per env."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_grad, compare_view, gpu_outputs  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def T(x, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)


def make_avatars(n_avatars, n_per, seed):
    avs = [synth.avatar_canonical(n_per, seed + k) for k in range(n_avatars)]
    av = {k: np.concatenate([a[k] for a in avs]) for k in avs[0]}
    G = np.stack([synth.random_pose(seed + k) for k in range(n_avatars)]).astype(np.float32)
    avatar_of = np.repeat(np.arange(n_avatars), n_per).astype(np.int32)
    return av, G, avatar_of


def gpu_avatars(api, av, avatar_of, n_avatars, dest=None):
    return api.Avatars(T(av["means"]), T(av["log_scales"]), T(av["quats"]), T(av["joint_ids"].view(np.int16),
                       torch.int16), T(av["weights"]), T(avatar_of, torch.int32), n_avatars, 24,
                       dest=None if dest is None else T(dest, torch.int64))


def test_deform_matches_oracle(gs, oracle):
    av, G, avatar_of = make_avatars(8, 5000, 0)
    m = av["means"].shape[0]
    A = gpu_avatars(gs, av, avatar_of, 8)
    om = torch.empty((m, 3), device="cuda")
    oc = torch.empty((m, 6), device="cuda")
    gs.deform(A, T(G), om, oc)
    torch.cuda.synchronize()
    pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32), av["weights"],
                        avatar_of, G.astype(np.float64))
    np.testing.assert_allclose(om.cpu().numpy(), pm, rtol=0, atol=2e-6 * (np.abs(pm).max() + 1))
    cov = oc.cpu().numpy()
    scale = np.abs(pc).max(axis=1, keepdims=True)
    assert np.abs(cov - pc).max() / scale.max() < 1e-5
    assert (np.abs(cov - pc) / scale).max() < 1e-4


def test_deform_scatter_by_dest(gs, oracle):
    av, G, avatar_of = make_avatars(2, 1000, 5)
    m = av["means"].shape[0]
    dest = np.random.default_rng(0).permutation(m + 500)[:m].astype(np.int64)
    A = gpu_avatars(gs, av, avatar_of, 2, dest)
    om = torch.zeros((m + 500, 3), device="cuda")
    oc = torch.zeros((m + 500, 6), device="cuda")
    gs.deform(A, T(G), om, oc)
    pm, _ = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32), av["weights"],
                       avatar_of, G.astype(np.float64))
    np.testing.assert_allclose(om.cpu().numpy()[dest], pm, atol=2e-5)
    untouched = np.setdiff1d(np.arange(m + 500), dest)
    assert torch.all(om[T(untouched, torch.int64)] == 0)


def test_deform_backward_matches_oracle(gs, oracle):
    av, G, avatar_of = make_avatars(3, 4000, 9)
    m = av["means"].shape[0]
    rng = np.random.default_rng(1)
    gm = rng.standard_normal((m, 3)).astype(np.float32)
    gc = rng.standard_normal((m, 6)).astype(np.float32) * 100.0
    A = gpu_avatars(gs, av, avatar_of, 3)
    grads = dict(means=torch.zeros((m, 3), device="cuda"), log_scales=torch.zeros((m, 3), device="cuda"),
                 quats=torch.zeros((m, 4), device="cuda"), G=torch.zeros((3, 24, 3, 4), device="cuda"))
    gs.deform_backward(A, T(G), T(gm), T(gc), grads)
    torch.cuda.synchronize()
    ref = oracle.lbs_backward(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32),
                              av["weights"], avatar_of, G.astype(np.float64), gm, gc)
    for k in ("means", "log_scales", "quats", "G"):
        check_grad(grads[k].cpu().numpy(), ref[k], f"LBS adjoint {k}", 1e-5)


def test_rooms_with_avatars_batched_vs_oracle(gs, oracle):
    # two envs: each a room plus 3 avatars posed inside it, deformed into the
    # concatenated arrays and rendered jointly with the scene in one pass
    W = H = 128
    envs, cams = [], []
    n_room, n_av, n_avatars = 60_000, 3000, 3
    for e in range(2):
        room = synth.room_scene(n_room, seed=300 + e)
        av, G, avatar_of = make_avatars(n_avatars, n_av, 40 + 10 * e)
        cam = synth.room_camera(300 + e, W, H)
        # place the avatars 2-3 m in front of the camera
        fwd, C = cam[6:9], cam[9:12]
        for k in range(n_avatars):
            root = C + fwd * (2.0 + 0.5 * k) + np.array([0.0, 0.0, -0.3])
            G[k, :, :, 3] += (root - G[k, 0, :, 3] - G[k, 0, :, :3] @ synth.REST_JOINTS[0]).astype(np.float32)
        envs.append((room, av, G, avatar_of))
        cams.append(cam)
    cams = np.stack(cams)
    # layout: env0 room, env0 avatars, env1 room, env1 avatars
    m_env = n_room + n_av * n_avatars
    offs = np.array([0, m_env, 2 * m_env])
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    cat = {k: np.concatenate([np.concatenate([r[k], a[k]]) for r, a, _, _ in envs]) for k in keys}
    dest = np.concatenate([np.arange(n_room, m_env) + e * m_env for e in range(2)]).astype(np.int64)
    av_all = {k: np.concatenate([a[k] for _, a, _, _ in envs]) for k in envs[0][1]}
    G_all = np.concatenate([G for _, _, G, _ in envs])
    avatar_of_all = np.concatenate([ao + n_avatars * e for e, (_, _, _, ao) in enumerate(envs)]).astype(np.int32)
    A = gpu_avatars(gs, av_all, avatar_of_all, 2 * n_avatars, dest)
    Gg = gs.Gaussians.from_numpy(dict(cat, cov3d=np.zeros((2 * m_env, 6), np.float32)))
    gs.deform(A, T(G_all), Gg.means, Gg.cov3d)
    r = gs.Renderer(gs.Batch(offs, env_cov3d_begin=[n_room, m_env + n_room]), W, H, persistent=True)
    out = r.forward(Gg, gs.cameras_tensor(cams))
    torch.cuda.synchronize()
    for e, (room, av, G, avatar_of) in enumerate(envs):
        pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32),
                            av["weights"], avatar_of, G.astype(np.float64))
        ge = {k: np.concatenate([room[k], av[k]]).astype(np.float64) for k in keys}
        ge["means"][n_room:] = pm
        ge["cov3d"] = np.concatenate([np.zeros((n_room, 6)), pc])
        ge["use_cov"] = np.concatenate([np.zeros(n_room, np.uint8), np.ones(len(pm), np.uint8)])
        ge["inexact"] = ge["use_cov"]
        ora = oracle.render(ge, cams[e], W, H)
        st = compare_view(gpu_outputs(out, e), ora)
        print(f"env {e} with avatars: {st}")
        assert (ora["T"] < 0.5).mean() > 0.1


def test_fused_lbs_in_preprocess_equals_deform_then_render(gs, oracle):
    """gs_render_avatars (LBS inside the preprocess, posed Gaussians never in
    memory) against gs_deform_avatars + gs_render on the same inputs, and
    against the oracle; gs_render_avatars_backward against gs_render_backward +
    gs_deform_avatars_backward."""
    W = H = 96
    n_room, n_av, n_avatars = 40_000, 3000, 2
    envs, cams = [], []
    for e in range(2):
        room = synth.room_scene(n_room, seed=700 + e)
        av, G, avatar_of = make_avatars(n_avatars, n_av, 80 + 10 * e)
        cam = synth.room_camera(700 + e, W, H)
        fwd, C = cam[6:9], cam[9:12]
        for k in range(n_avatars):
            root = C + fwd * (2.0 + 0.6 * k) + np.array([0.0, 0.0, -0.3])
            G[k, :, :, 3] += (root - G[k, 0, :, 3] - G[k, 0, :, :3] @ synth.REST_JOINTS[0]).astype(np.float32)
        envs.append((room, av, G, avatar_of))
        cams.append(cam)
    cams = np.stack(cams)
    m_env = n_room + n_av * n_avatars
    offs = np.array([0, m_env, 2 * m_env])
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    cat = {k: np.concatenate([np.concatenate([r[k], a[k]]) for r, a, _, _ in envs]) for k in keys}
    dest = np.concatenate([np.arange(n_room, m_env) + e * m_env for e in range(2)]).astype(np.int64)
    av_all = {k: np.concatenate([a[k] for _, a, _, _ in envs]) for k in envs[0][1]}
    G_all = T(np.concatenate([G for _, _, G, _ in envs]))
    avatar_of_all = np.concatenate([ao + n_avatars * e for e, (_, _, _, ao) in enumerate(envs)]).astype(np.int32)
    batch = gs.Batch(offs, env_cov3d_begin=[n_room, m_env + n_room])
    # unfused: deform into the rows, then render
    Gg = gs.Gaussians.from_numpy(dict(cat, cov3d=np.zeros((2 * m_env, 6), np.float32)))
    gs.deform(gpu_avatars(gs, av_all, avatar_of_all, 2 * n_avatars, dest), G_all, Gg.means, Gg.cov3d)
    r1 = gs.Renderer(batch, W, H, persistent=True)
    ct = gs.cameras_tensor(cams)
    a = [x.clone() for x in r1.forward(Gg, ct)]
    # fused: the avatar rows of `cat` keep their canonical (unposed) values
    Gf = gs.Gaussians.from_numpy(cat)
    r2 = gs.Renderer(batch, W, H, persistent=True)
    av_f = gpu_avatars(gs, av_all, avatar_of_all, 2 * n_avatars)
    b = r2.forward_avatars(Gf, av_f, G_all, ct)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # the adjoints: gs_render_backward + gs_deform_avatars_backward against
    # gs_render_avatars_backward, equal up to the order of float atomics
    rng = np.random.default_rng(5)
    d_rgb = T(rng.standard_normal((2, 3, H, W)))
    d_depth = T(0.1 * rng.standard_normal((2, H, W)))
    g1 = r1.backward(Gg, ct, d_rgb, d_depth)
    ga1 = dict(means=torch.zeros((2 * n_avatars * n_av, 3), device="cuda"),
               log_scales=torch.zeros((2 * n_avatars * n_av, 3), device="cuda"),
               quats=torch.zeros((2 * n_avatars * n_av, 4), device="cuda"), G=torch.zeros_like(G_all))
    gs.deform_backward(gpu_avatars(gs, av_all, avatar_of_all, 2 * n_avatars, dest), G_all, g1["means"], g1["cov3d"],
                       ga1)
    g2, ga2 = r2.backward_avatars(Gf, av_f, G_all, ct, d_rgb, d_depth)
    torch.cuda.synchronize()
    assert r2.status() == 0
    av_rows = torch.from_numpy(dest).cuda()
    pairs = [(g1[k], g2[k], k) for k in ("means", "opacity_logits", "sh")]
    pairs += [(g1["cov3d"][av_rows], g2["cov3d"][av_rows], "posed cov3d")]
    pairs += [(ga1[k], ga2[k], "canonical " + k) for k in ("means", "log_scales", "quats", "G")]
    scene_rows = torch.ones(2 * m_env, dtype=torch.bool, device="cuda")
    scene_rows[av_rows] = False
    pairs += [(g1[k][scene_rows], g2[k][scene_rows], "scene " + k) for k in ("log_scales", "quats")]
    for x, y, name in pairs:
        scale = float(x.abs().max())
        assert scale > 0, name
        err = float((x - y).abs().max())
        assert err <= 1e-5 * scale, (name, err, scale)
    for e, (room, av, G, avatar_of) in enumerate(envs):
        pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32),
                            av["weights"], avatar_of, G.astype(np.float64))
        ge = {k: np.concatenate([room[k], av[k]]).astype(np.float64) for k in keys}
        ge["means"][n_room:] = pm
        ge["cov3d"] = np.concatenate([np.zeros((n_room, 6)), pc])
        ge["use_cov"] = np.concatenate([np.zeros(n_room, np.uint8), np.ones(len(pm), np.uint8)])
        ge["inexact"] = ge["use_cov"]
        compare_view(gpu_outputs(b, e), oracle.render(ge, cams[e], W, H))


def test_fused_lbs_rejects_bad_layouts(gs):
    W = H = 32
    room = synth.room_scene(2000, seed=1)
    av, G, avatar_of = make_avatars(1, 500, 3)
    cat = {k: np.concatenate([room[k], av[k]]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    n = cat["means"].shape[0]
    Gf = gs.Gaussians.from_numpy(cat)
    ct = gs.cameras_tensor(synth.room_camera(1, W, H)[None])
    A = gpu_avatars(gs, av, avatar_of, 1)
    r = gs.Renderer(gs.Batch(np.array([0, n]), env_cov3d_begin=[2000 + 1]), W, H)  # 499 rows, 500 canonical
    with pytest.raises(gs.GsError, match="INVALID_ARG"):
        r.forward_avatars(Gf, A, T(G), ct)
    r = gs.Renderer(gs.Batch(np.array([0, n])), W, H)  # no avatar rows declared
    with pytest.raises(gs.GsError, match="INVALID_ARG"):
        r.forward_avatars(Gf, A, T(G), ct)


def test_fused_lbs_canonical_sh_direction(gs, oracle):
    """GS_FLAG_AVATAR_CANONICAL_SH: the avatars' SH evaluated at A3^-1 (mu' - C)
    against the oracle with that direction matrix; it differs from the world
    direction render wherever the avatars show."""
    W = H = 96
    n_room, n_av, n_avatars = 20_000, 4000, 2
    room = synth.room_scene(n_room, seed=810)
    av, G, avatar_of = make_avatars(n_avatars, n_av, 90)
    av["sh"][:, 1:4] += np.random.default_rng(5).normal(0, 0.4, (n_av * n_avatars, 3, 3)).astype(np.float32)
    cam = synth.room_camera(810, W, H)
    fwd, C = cam[6:9], cam[9:12]
    for k in range(n_avatars):
        root = C + fwd * (1.8 + 0.6 * k) + np.array([0.0, 0.0, -0.3])
        G[k, :, :, 3] += (root - G[k, 0, :, 3]).astype(np.float32)
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    cat = {k: np.concatenate([room[k], av[k]]) for k in keys}
    n = cat["means"].shape[0]
    batch = gs.Batch(np.array([0, n]), env_cov3d_begin=[n_room])
    A = gpu_avatars(gs, av, avatar_of, n_avatars)
    ct = gs.cameras_tensor(cam[None])
    r = gs.Renderer(batch, W, H)
    world = [x.clone() for x in r.forward_avatars(gs.Gaussians.from_numpy(cat), A, T(G), ct)]
    r.cfg.flags |= gs.FLAG_AVATAR_CANONICAL_SH
    canon = r.forward_avatars(gs.Gaussians.from_numpy(cat), A, T(G), ct)
    torch.cuda.synchronize()
    ids = av["joint_ids"].astype(np.int32)
    pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], ids, av["weights"], avatar_of,
                        G.astype(np.float64))
    Am = oracle.lbs_matrices(ids, av["weights"], avatar_of, G.astype(np.float64))
    dirmat = np.concatenate([np.tile(np.eye(3).reshape(1, 9), (n_room, 1)),
                             np.linalg.inv(Am[:, :, :3]).reshape(-1, 9)])
    ge = {k: cat[k].astype(np.float64) for k in keys}
    ge["means"][n_room:] = pm
    ge.update(cov3d=np.concatenate([np.zeros((n_room, 6)), pc]),
              use_cov=np.concatenate([np.zeros(n_room, np.uint8), np.ones(len(pm), np.uint8)]))
    ge["inexact"] = ge["use_cov"]
    compare_view(gpu_outputs(canon, 0), oracle.render(dict(ge, sh_dirmat=dirmat), cam, W, H))
    assert not torch.equal(world[0], canon[0])  # the canonical direction changes the avatars' colour
    assert torch.equal(world[1], canon[1])  # and nothing else
