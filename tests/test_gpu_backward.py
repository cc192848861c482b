"""Adjoint of the CUDA path (gs_render_backward, gs_deform_avatars_backward,
the autograd Functions) against the FP64 oracle adjoint, which is itself pinned
to FP64 central finite differences (tests/test_oracle_adjoint.py).  Every
parameter group is checked by its relative L2 error and element by element
(|g - g_oracle| <= 1e-3 max|g_oracle| + 1e-7, the worst element reported).
Room scenes pass no upstream gradient through the pixels the oracle flags as
ambiguous: there an FP32 decision may legitimately differ from the FP64 one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_grad  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def mask_ambiguous(oracle, g, cams, W, H, d_rgb, d_depth, offs=None, view_env=None):
    """Zero the upstream gradient at every pixel the oracle flags (in place)."""
    n = g["means"].shape[0]
    offs = np.array([0, n]) if offs is None else offs
    view_env = np.arange(len(offs) - 1) if view_env is None else np.asarray(view_env)
    flagged = 0
    for v, e in enumerate(view_env):
        sl = slice(offs[e], offs[e + 1])
        amb = oracle.render({k: x[sl] for k, x in g.items()}, cams[v], W, H)["amb"] != 0
        d_rgb[v][:, amb] = 0.0
        d_depth[v][amb] = 0.0
        flagged += int(amb.sum())
    return flagged


def gpu_forward_backward(api, g, cams, W, H, d_rgb, d_depth, offs=None, view_env=None, sh_dtype=torch.float32, **kw):
    n = g["means"].shape[0]
    offs = np.array([0, n]) if offs is None else offs
    r = api.Renderer(api.Batch(offs, view_env), W, H, **kw)
    G = api.Gaussians.from_numpy(g, sh_dtype=sh_dtype)
    ct = api.cameras_tensor(cams)
    r.forward(G, ct)
    gr = r.backward(G, ct, torch.from_numpy(d_rgb).float().cuda(), torch.from_numpy(d_depth).float().cuda())
    torch.cuda.synchronize()
    assert r.status() == 0
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in gr.items()}


def oracle_grads(oracle, g, cams, W, H, d_rgb, d_depth, offs=None, view_env=None):
    n = g["means"].shape[0]
    offs = np.array([0, n]) if offs is None else offs
    view_env = np.arange(len(offs) - 1) if view_env is None else np.asarray(view_env)
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logits=np.zeros(n), sh=np.zeros((n, 16, 3)))
    for v, e in enumerate(view_env):
        sl = slice(offs[e], offs[e + 1])
        ge = {k: x[sl] for k, x in g.items()}
        gv = oracle.render_backward(ge, cams[v], W, H, d_rgb[v], d_depth[v])
        for k in GROUPS:
            out[k][sl] += gv[k]
    return out


def test_backward_matches_oracle_box_scene(gs, oracle):
    g = synth.box_scene(3000, seed=0)
    g["log_scales"] += np.float32(0.7)
    W = H = 96
    cam = synth.identity_camera(W, H)
    rng = np.random.default_rng(0)
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = rng.standard_normal((1, H, W)).astype(np.float32)
    a = gpu_forward_backward(gs, g, cam[None], W, H, d_rgb, d_depth)
    b = oracle_grads(oracle, g, cam[None], W, H, d_rgb, d_depth)
    for k in GROUPS:
        check_grad(a[k], b[k], f"box {k}", 1e-4)


def test_backward_matches_oracle_room_views(gs, oracle):
    g = synth.room_scene(120_000, seed=3)
    W = H = 128
    cams = np.stack([synth.room_camera(30 + k, W, H) for k in range(3)])
    rng = np.random.default_rng(1)
    d_rgb = rng.standard_normal((3, 3, H, W)).astype(np.float32)
    d_depth = (0.1 * rng.standard_normal((3, H, W))).astype(np.float32)
    offs = np.array([0, 120_000])
    mask_ambiguous(oracle, g, cams, W, H, d_rgb, d_depth, offs=offs, view_env=[0, 0, 0])
    a = gpu_forward_backward(gs, g, cams, W, H, d_rgb, d_depth, offs=offs, view_env=[0, 0, 0])
    b = oracle_grads(oracle, g, cams, W, H, d_rgb, d_depth, offs=offs, view_env=[0, 0, 0])
    for k in GROUPS:
        check_grad(a[k], b[k], f"room {k}", 1e-3)


def test_backward_batched_envs_and_persistent(gs, oracle):
    g, offs, cams = synth.batched_rooms(n_envs=3, n_min=20_000, n_max=60_000, W=96, H=96, seed0=200)
    W = H = 96
    rng = np.random.default_rng(2)
    d_rgb = rng.standard_normal((3, 3, H, W)).astype(np.float32)
    d_depth = (0.1 * rng.standard_normal((3, H, W))).astype(np.float32)
    mask_ambiguous(oracle, g, cams, W, H, d_rgb, d_depth, offs=offs)
    a = gpu_forward_backward(gs, g, cams, W, H, d_rgb, d_depth, offs=offs, persistent=True)
    b = oracle_grads(oracle, g, cams, W, H, d_rgb, d_depth, offs=offs)
    for k in GROUPS:
        check_grad(a[k], b[k], f"batched {k}", 1e-3)


@pytest.mark.parametrize("tile,depth,pix", [((8, 8), 64, (1, 1)), ((16, 16), 256, (2, 2)), ((16, 8), 128, (2, 1)),
                                            ((8, 16), 64, (1, 2))])
def test_backward_tile_and_pixels_per_thread(gs, oracle, tile, depth, pix):
    g = synth.room_scene(80_000, seed=9)
    W, H = 136, 104  # ragged against every tile
    cam = synth.room_camera(9, W, H)
    rng = np.random.default_rng(5)
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = (0.1 * rng.standard_normal((1, H, W))).astype(np.float32)
    mask_ambiguous(oracle, g, cam[None], W, H, d_rgb, d_depth)
    a = gpu_forward_backward(gs, g, cam[None], W, H, d_rgb, d_depth, tile=tile, batch_depth=depth, pix=pix)
    b = oracle_grads(oracle, g, cam[None], W, H, d_rgb, d_depth)
    for k in GROUPS:
        check_grad(a[k], b[k], f"tile {tile} pix {pix} {k}", 1e-3)


@pytest.mark.parametrize("persistent", [False, True])
def test_backward_heavy_tiles_split_into_segments(gs, oracle, persistent):
    # a dense room seen at 64x64: tiles hold several thousand pairs, so the
    # backward runs them as 2048-long segments started from forward checkpoints
    g = synth.room_scene(400_000, seed=12)
    W = H = 64
    cam = synth.room_camera(12, W, H)
    rng = np.random.default_rng(6)
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = (0.1 * rng.standard_normal((1, H, W))).astype(np.float32)
    mask_ambiguous(oracle, g, cam[None], W, H, d_rgb, d_depth)
    r = gs.Renderer(gs.Batch(np.array([0, 400_000])), W, H, persistent=persistent)
    G = gs.Gaussians.from_numpy(g)
    ct = gs.cameras_tensor(cam[None])
    r.forward(G, ct)
    st = r.stats()
    assert st["max_bin"] > 3 * 2048, st
    gr = r.backward(G, ct, torch.from_numpy(d_rgb).cuda(), torch.from_numpy(d_depth).cuda())
    torch.cuda.synchronize()
    b = oracle_grads(oracle, g, cam[None], W, H, d_rgb, d_depth)
    for k in GROUPS:
        check_grad(gr[k].cpu().numpy(), b[k], f"heavy-tile {k}", 1e-3)


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_backward_half_sh(gs, oracle, dt):
    g = synth.box_scene(2000, seed=4)
    g["log_scales"] += np.float32(0.7)
    W = H = 64
    cam = synth.identity_camera(W, H)
    rng = np.random.default_rng(3)
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = rng.standard_normal((1, H, W)).astype(np.float32)
    tdt = torch.float16 if dt == "f16" else torch.bfloat16
    a = gpu_forward_backward(gs, g, cam[None], W, H, d_rgb, d_depth, sh_dtype=tdt)
    gq = dict(g)
    gq["sh"] = (g["sh"].astype(np.float16).astype(np.float32) if dt == "f16"
                else synth.bf16_to_f32(synth.bf16_bits(g["sh"])))
    b = oracle_grads(oracle, gq, cam[None], W, H, d_rgb, d_depth)
    for k in GROUPS:
        check_grad(a[k], b[k], f"{dt} SH {k}", 1e-4)


def test_autograd_function_l1_loss(gs):
    g = synth.box_scene(2000, seed=5)
    g["log_scales"] += np.float32(0.7)
    W = H = 64
    cam = synth.identity_camera(W, H)
    r = gs.Renderer(gs.Batch(np.array([0, 2000])), W, H)
    ct = gs.cameras_tensor(cam[None])
    params = {k: torch.from_numpy(np.ascontiguousarray(g[k])).cuda().requires_grad_(True)
              for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    target = torch.rand((1, 3, H, W), device="cuda")
    rgb, depth = gs.render(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                           params["sh"], r, ct)
    loss = (rgb - target).abs().mean() + 0.1 * depth.mean()
    loss.backward()
    d_rgb = (torch.sign(rgb - target) / rgb.numel()).detach()
    d_depth = torch.full_like(depth, 0.1 / depth.numel())
    G = gs.Gaussians(*(params[k].detach() for k in ("means", "log_scales", "quats", "opacity_logits", "sh")))
    r2 = gs.Renderer(gs.Batch(np.array([0, 2000])), W, H)
    r2.forward(G, ct)
    ref = r2.backward(G, ct, d_rgb, d_depth)
    # two backward runs: the record gradients are summed with float atomics in
    # whatever order the tiles finish, so they agree to rounding relative to the
    # largest gradient of the group, not element by element
    for k in params:
        torch.testing.assert_close(params[k].grad, ref[k], rtol=1e-5, atol=1e-6 * float(ref[k].abs().max()))


def _avatar_scene(seed, n_scene=100, n_av=100, n_avatars=2):
    rng = np.random.default_rng(seed)
    sc = synth.box_scene(n_scene, seed=seed)
    sc["log_scales"] = rng.normal(-1.6, 0.3, (n_scene, 3)).astype(np.float32)
    avs = [synth.avatar_canonical(n_av, seed + k) for k in range(n_avatars)]
    av = {k: np.concatenate([a[k] for a in avs]) for k in avs[0]}
    av["means"] *= np.float32(0.4)
    av["log_scales"] = rng.normal(-2.3, 0.3, (n_av * n_avatars, 3)).astype(np.float32)
    Gm = np.stack([synth.random_pose(seed + k, root_t=[0.3 * k - 0.15, 0.0, 3.0]) for k in range(n_avatars)])
    # keep the avatars in front of the camera: undo the random root yaw's translation drift
    Gm = Gm.astype(np.float32)
    avatar_of = np.repeat(np.arange(n_avatars), n_av).astype(np.int32)
    return sc, av, Gm, avatar_of


def test_scene_with_avatars_forward_backward_vs_oracle(gs, oracle):
    sc, av, Gm, avatar_of = _avatar_scene(11)
    ns, m = sc["means"].shape[0], av["means"].shape[0]
    W = H = 48
    cam = synth.identity_camera(W, H)
    # oracle: FP64 LBS then render, adjoint through both
    pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32), av["weights"],
                        avatar_of, Gm.astype(np.float64))
    gall = dict(means=np.concatenate([sc["means"].astype(np.float64), pm]),
                log_scales=np.concatenate([sc["log_scales"], np.zeros((m, 3), np.float32)]),
                quats=np.concatenate([sc["quats"], np.tile(np.float32([1, 0, 0, 0]), (m, 1))]),
                opacity_logits=np.concatenate([sc["opacity_logits"], av["opacity_logits"]]),
                sh=np.concatenate([sc["sh"], av["sh"]]), cov3d=np.concatenate([np.zeros((ns, 6)), pc]),
                use_cov=np.concatenate([np.zeros(ns, np.uint8), np.ones(m, np.uint8)]),
                inexact=np.concatenate([np.zeros(ns, np.uint8), np.ones(m, np.uint8)]))
    ora = oracle.render(gall, cam, W, H)
    rng = np.random.default_rng(4)
    d_rgb = rng.standard_normal((3, H, W))
    d_depth = rng.standard_normal((H, W))
    og = oracle.render_backward(gall, cam, W, H, d_rgb, d_depth)
    oga = oracle.lbs_backward(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32),
                              av["weights"], avatar_of, Gm.astype(np.float64), og["means"][ns:], og["cov3d"][ns:])
    # GPU: autograd through SceneWithAvatarsFunction
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)  # noqa: E731
    sp = [T(sc[k]).requires_grad_(True) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    ap = [T(av[k]).requires_grad_(True) for k in ("means", "log_scales", "quats")]
    aop, ash = T(av["opacity_logits"]).requires_grad_(True), T(av["sh"]).requires_grad_(True)
    Gt = T(Gm).requires_grad_(True)
    static = (T(av["joint_ids"].view(np.int16), torch.int16), T(av["weights"]), T(avatar_of, torch.int32), 2, 24)
    r = gs.Renderer(gs.Batch(np.array([0, ns + m]), env_cov3d_begin=[ns]), W, H)
    rgb, depth = gs.SceneWithAvatarsFunction.apply(*sp, *ap, aop, ash, Gt, static, r, gs.cameras_tensor(cam[None]))
    from helpers import compare_view
    compare_view(dict(rgb=rgb[0].detach().cpu().numpy(), depth=depth[0].detach().cpu().numpy(),
                      T=ora["T"], n_contrib=ora["n_contrib"]), ora)
    loss = (rgb[0] * T(d_rgb)).sum() + (depth[0] * T(d_depth)).sum()
    loss.backward()
    pairs = [(sp[0].grad, og["means"][:ns]), (sp[1].grad, og["log_scales"][:ns]), (sp[2].grad, og["quats"][:ns]),
             (sp[3].grad, og["opacity_logits"][:ns]), (sp[4].grad, og["sh"][:ns]), (ap[0].grad, oga["means"]),
             (ap[1].grad, oga["log_scales"]), (ap[2].grad, oga["quats"]), (aop.grad, og["opacity_logits"][ns:]),
             (ash.grad, og["sh"][ns:]), (Gt.grad, oga["G"])]
    names = ("scene means", "scene log_scales", "scene quats", "scene opacity_logits", "scene sh", "avatar means",
             "avatar log_scales", "avatar quats", "avatar opacity_logits", "avatar sh", "joint G")
    for name, (a, b) in zip(names, pairs):
        check_grad(a.cpu().numpy(), b, f"avatar-scene {name}", 1e-3)


def test_repeated_backward_of_one_forward(gs):
    """Two backward calls after one forward (as autograd with retain_graph
    does) give the same gradients: the record gradient rows the first call
    filled are cleared before the second accumulates into them; a new forward
    starts from clean rows again."""
    g = synth.room_scene(150_000, seed=21)
    W = H = 96
    cam = synth.room_camera(21, W, H)
    rng = np.random.default_rng(3)
    d_rgb = torch.from_numpy(rng.standard_normal((1, 3, H, W))).float().cuda()
    d_dep = torch.from_numpy(0.1 * rng.standard_normal((1, H, W))).float().cuda()
    r = gs.Renderer(gs.Batch(np.array([0, g["means"].shape[0]])), W, H, tile=(8, 8), batch_depth=64, pix=(2, 1),
                    persistent=True, grad_overwrite=True)
    G = gs.Gaussians.from_numpy(g)
    ct = gs.cameras_tensor(cam[None])
    r.forward(G, ct)
    a = {k: v.clone() for k, v in r.backward(G, ct, d_rgb, d_dep).items() if v is not None}
    b = {k: v.clone() for k, v in r.backward(G, ct, d_rgb, d_dep).items() if v is not None}
    r.forward(G, ct)
    c = {k: v.clone() for k, v in r.backward(G, ct, d_rgb, d_dep).items() if v is not None}
    torch.cuda.synchronize()
    for k in a:  # equal up to the order of the float atomics (a stale row would double a gradient)
        check_grad(b[k].cpu().numpy(), a[k].cpu().numpy(), f"second backward {k}", 2e-5, 1e-5, 1e-9)
        check_grad(c[k].cpu().numpy(), a[k].cpu().numpy(), f"new forward {k}", 2e-5, 1e-5, 1e-9)
    assert float(a["opacity_logits"].abs().sum()) > 0


@pytest.mark.parametrize("overwrite", [False, True])
def test_backward_edge_cases(gs, oracle, overwrite):
    """Degenerate inputs of the adjoint, in both gradient modes: a scene the
    near plane culls entirely (every gradient exactly zero), an empty env next
    to a non-empty one at 1x1 pixels (hundreds of Gaussians through one pixel
    that stops), and one Gaussian covering a ragged 37x23 image, the last two
    against the oracle adjoint."""
    W, H = 37, 23
    cam = synth.identity_camera(W, H)
    rng = np.random.default_rng(40)
    kw = dict(grad_overwrite=overwrite)
    # everything behind the camera
    g = synth.box_scene(500, seed=10)
    g["means"][:, 2] = np.float32(-1.0)
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = rng.standard_normal((1, H, W)).astype(np.float32)
    a = gpu_forward_backward(gs, g, cam[None], W, H, d_rgb, d_depth, **kw)
    for k in GROUPS:
        assert np.all(a[k] == 0.0), k
    # an empty env next to a non-empty one; 1x1 image
    g = synth.box_scene(400, seed=11)
    g["log_scales"] += np.float32(2.0)
    offs = np.array([0, 0, 400])
    c1 = synth.identity_camera(1, 1)
    cams = np.stack([c1, c1])
    d_rgb = rng.standard_normal((2, 3, 1, 1)).astype(np.float32)
    d_depth = rng.standard_normal((2, 1, 1)).astype(np.float32)
    mask_ambiguous(oracle, g, cams, 1, 1, d_rgb, d_depth, offs=offs)
    a = gpu_forward_backward(gs, g, cams, 1, 1, d_rgb, d_depth, offs=offs, **kw)
    b = oracle_grads(oracle, g, cams, 1, 1, d_rgb, d_depth, offs=offs)
    assert np.abs(b["opacity_logits"]).max() > 0  # the pixel passes gradient
    for k in GROUPS:
        check_grad(a[k], b[k], f"1x1 {k}", 1e-3)
    # one Gaussian covering the whole image
    g = dict(means=np.float32([[0.1, -0.05, 3.0]]), log_scales=np.float32([[1.0, 0.8, 1.2]]),
             quats=np.float32([[0.9, 0.1, -0.2, 0.3]]), opacity_logits=np.float32([1.5]),
             sh=(0.3 * rng.standard_normal((1, 16, 3))).astype(np.float32))
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = rng.standard_normal((1, H, W)).astype(np.float32)
    mask_ambiguous(oracle, g, cam[None], W, H, d_rgb, d_depth)
    a = gpu_forward_backward(gs, g, cam[None], W, H, d_rgb, d_depth, **kw)
    b = oracle_grads(oracle, g, cam[None], W, H, d_rgb, d_depth)
    for k in GROUPS:
        check_grad(a[k], b[k], f"one Gaussian {k}", 1e-4)


def test_overwrite_mode_clears_unseen_rows(gs):
    """Overwrite mode (GS_FLAG_GRAD_OVERWRITE) on gradient buffers full of
    garbage: every row ends as the accumulate mode's gradient into zeroed
    buffers, the rows of Gaussians no view sees exactly zero.  N = 4001 makes
    every gradient array end off a 16-byte boundary (the clearing's scalar tail)."""
    n = 4001
    g = synth.box_scene(n, seed=31)
    g["means"][1::2, 2] = -g["means"][1::2, 2]  # every other Gaussian behind the camera: unseen
    W = H = 64
    cam = synth.identity_camera(W, H)
    rng = np.random.default_rng(31)
    d_rgb = torch.from_numpy(rng.standard_normal((1, 3, H, W))).float().cuda()
    d_dep = torch.from_numpy(0.1 * rng.standard_normal((1, H, W))).float().cuda()
    G = gs.Gaussians.from_numpy(g)
    ct = gs.cameras_tensor(cam[None])
    kw = dict(tile=(8, 8), batch_depth=64, pix=(2, 1), persistent=True)
    ref_r = gs.Renderer(gs.Batch(np.array([0, n])), W, H, **kw)
    ref_r.forward(G, ct)
    ref = ref_r.backward(G, ct, d_rgb, d_dep)  # accumulate into zeros
    r = gs.Renderer(gs.Batch(np.array([0, n])), W, H, grad_overwrite=True, **kw)
    r.forward(G, ct)
    junk = dict(means=torch.full((n, 3), 7.0, device="cuda"), log_scales=torch.full((n, 3), -3.0, device="cuda"),
                quats=torch.full((n, 4), 5.0, device="cuda"), opacity_logits=torch.full((n,), 9.0, device="cuda"),
                sh=torch.full((n, 16, 3), 11.0, device="cuda"))
    out = r.backward(G, ct, d_rgb, d_dep, grads=junk)
    torch.cuda.synchronize()
    for k in GROUPS:
        a, b = out[k].cpu().numpy(), ref[k].cpu().numpy()
        assert np.all(a[1::2] == 0.0), k  # unseen rows cleared
        check_grad(a, b, f"overwrite {k}", 2e-5, 1e-5, 1e-9)
    assert float(ref["opacity_logits"].abs().sum()) > 0


def test_precleared_mode_after_zero_gradients_on_a_side_stream(gs):
    """gs_zero_gradients on a second stream beside the forward, joined by an
    event, then the backward with GS_FLAG_GRAD_PRECLEARED: the overwrite mode's
    result (buffers full of garbage before, unseen rows exactly zero), with
    arrays ending off a 16-byte boundary (N = 4001)."""
    n = 4001
    g = synth.box_scene(n, seed=32)
    g["means"][1::2, 2] = -g["means"][1::2, 2]  # every other Gaussian behind the camera: unseen
    W = H = 64
    cam = synth.identity_camera(W, H)
    rng = np.random.default_rng(32)
    d_rgb = torch.from_numpy(rng.standard_normal((1, 3, H, W))).float().cuda()
    d_dep = torch.from_numpy(0.1 * rng.standard_normal((1, H, W))).float().cuda()
    G = gs.Gaussians.from_numpy(g)
    ct = gs.cameras_tensor(cam[None])
    kw = dict(tile=(8, 8), batch_depth=64, pix=(2, 1), persistent=True)
    ref_r = gs.Renderer(gs.Batch(np.array([0, n])), W, H, **kw)
    ref_r.forward(G, ct)
    ref = ref_r.backward(G, ct, d_rgb, d_dep)  # accumulate into zeros
    r = gs.Renderer(gs.Batch(np.array([0, n])), W, H, grad_overwrite=True, **kw)
    junk = dict(means=torch.full((n, 3), 7.0, device="cuda"), log_scales=torch.full((n, 3), -3.0, device="cuda"),
                quats=torch.full((n, 4), 5.0, device="cuda"), opacity_logits=torch.full((n,), 9.0, device="cuda"),
                sh=torch.full((n, 16, 3), 11.0, device="cuda"), cov3d=torch.full((n, 6), 2.0, device="cuda"))
    main, side = torch.cuda.Stream(), torch.cuda.Stream()
    main.wait_stream(torch.cuda.current_stream())
    side.wait_stream(torch.cuda.current_stream())
    gs.zero_gradients(junk, n_ctas=3, stream=side)
    cleared = torch.cuda.Event()
    cleared.record(side)
    r.forward(G, ct, stream=main)
    main.wait_event(cleared)
    out = r.backward(G, ct, d_rgb, d_dep, grads=junk, stream=main, precleared=True)
    torch.cuda.synchronize()
    assert float(out["cov3d"].abs().max()) == 0.0  # no Gaussian takes cov3d: cleared, never written
    for k in GROUPS:
        a, b = out[k].cpu().numpy(), ref[k].cpu().numpy()
        assert np.all(a[1::2] == 0.0), k
        check_grad(a, b, f"precleared {k}", 2e-5, 1e-5, 1e-9)
    assert float(ref["opacity_logits"].abs().sum()) > 0
