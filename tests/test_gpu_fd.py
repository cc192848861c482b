"""The CUDA adjoint against FP64 central finite differences of the oracle's
forward, on the finite-difference case: 100 scene Gaussians and a 100-Gaussian
avatar posed by LBS (24 joints), one 32x32 view with f = 16.  The gradients of
L = <w_rgb, rgb> + <w_d, depth> with respect to every scene and avatar
parameter and the joint transforms come from gs_deform_avatars, gs_render,
gs_render_backward and gs_deform_avatars_backward: through the autograd
SceneWithAvatarsFunction with FP32 SH, through api.AvatarScene (FP32 gradient
buffers) with FP16 SH.  The inputs are FP32 values and the differences are
taken at those values (step 1e-4 max(|x|, 1), FP64, so that the differences'
own rounding stays far below the smallest gradients); pixels the oracle flags
as ambiguous carry no weight, on both sides.  Per group, on the sampled
coordinates: relative L2 <= 1e-3 and |g - g_fd| <= 1e-3 max|g_fd| + 1e-7 (the
differentiable rasterisation of Sec. 2.2 / Sec. 3.2, avatars of Sec. 3.3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from fd_case import W, H, as64, central_differences, fd_camera, fd_scene, posed_scene  # noqa: E402
from helpers import check_grad  # noqa: E402

H_REL = 1e-4


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def _autograd_grads(gs, sc32, av32, G, cam, wr, wd):
    ns, m = len(sc32["means"]), len(av32["means"])
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)  # noqa: E731
    sp = [T(sc32[k]).requires_grad_(True) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    ap = [T(av32[k]).requires_grad_(True) for k in ("means", "log_scales", "quats")]
    aop = T(av32["opacity_logits"]).requires_grad_(True)
    ash = T(av32["sh"]).requires_grad_(True)
    Gt = T(G).requires_grad_(True)
    static = (T(av32["joint_ids"].view(np.int16), torch.int16), T(av32["weights"]),
              T(np.zeros(m, np.int32), torch.int32), 1, 24)
    r = gs.Renderer(gs.Batch(np.array([0, ns + m]), env_cov3d_begin=[ns]), W, H)
    rgb, depth = gs.SceneWithAvatarsFunction.apply(*sp, *ap, aop, ash, Gt, static, r, gs.cameras_tensor(cam[None]))
    loss = (rgb[0] * T(wr)).sum() + (depth[0] * T(wd)).sum()
    loss.backward()
    torch.cuda.synchronize()
    return {("sc", "means"): sp[0].grad, ("sc", "log_scales"): sp[1].grad, ("sc", "quats"): sp[2].grad,
            ("sc", "opacity_logits"): sp[3].grad, ("sc", "sh"): sp[4].grad, ("av", "means"): ap[0].grad,
            ("av", "log_scales"): ap[1].grad, ("av", "quats"): ap[2].grad, ("av", "opacity_logits"): aop.grad,
            ("av", "sh"): ash.grad, ("G", "G"): Gt.grad}


def _avatar_scene_grads(gs, sc32, av32, G, cam, wr, wd, sh_dtype):
    ns = len(sc32["means"])
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)  # noqa: E731
    scene = {k: T(sc32[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    avatars = {k: T(av32[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "weights")}
    avatars["joint_ids"] = T(av32["joint_ids"].view(np.int16), torch.int16)
    avatars["avatar_of"] = T(np.zeros(len(av32["means"]), np.int32), torch.int32)
    sc = gs.AvatarScene(scene, avatars, 1, 24, W, H, 1, sh_dtype=sh_dtype)
    Gt = T(G)
    ct = gs.cameras_tensor(cam[None])
    sc.forward(Gt, ct)
    gr, ga = sc.backward(Gt, ct, T(wr[None]), T(wd[None]))
    torch.cuda.synchronize()
    return {("sc", "means"): gr["means"][:ns], ("sc", "log_scales"): gr["log_scales"][:ns],
            ("sc", "quats"): gr["quats"][:ns], ("sc", "opacity_logits"): gr["opacity_logits"][:ns],
            ("sc", "sh"): gr["sh"][:ns], ("av", "means"): ga["means"], ("av", "log_scales"): ga["log_scales"],
            ("av", "quats"): ga["quats"], ("av", "opacity_logits"): gr["opacity_logits"][ns:],
            ("av", "sh"): gr["sh"][ns:], ("G", "G"): ga["G"]}


@pytest.mark.parametrize("path", ["autograd_f32_sh", "avatar_scene_f16_sh"])
def test_cuda_adjoint_matches_fp64_finite_differences(gs, oracle, path):
    sc32, av32, G = fd_scene()
    G = G.astype(np.float32).astype(np.float64)  # the joint transforms the GPU reads
    if path.endswith("f16_sh"):  # differences at the stored SH values
        sc32["sh"] = sc32["sh"].astype(np.float16).astype(np.float32)
        av32["sh"] = av32["sh"].astype(np.float16).astype(np.float32)
    sc, av = as64(sc32), as64(av32)
    cam = fd_camera()
    rng = np.random.default_rng(7)
    wr = rng.standard_normal((3, H, W))
    wd = rng.standard_normal((H, W))
    g = posed_scene(oracle, sc, av, G)
    g["inexact"] = g["use_cov"]  # posed by FP32 LBS on the GPU
    ora = oracle.render(g, cam, W, H)
    assert (ora["T"] < 0.9).mean() > 0.2
    amb = ora["amb"] != 0
    wr[:, amb] = 0.0
    wd[amb] = 0.0
    if path == "autograd_f32_sh":
        cuda = _autograd_grads(gs, sc32, av32, G, cam, wr, wd)
    else:
        cuda = _avatar_scene_grads(gs, sc32, av32, G, cam, wr, wd, torch.float16)
    checked = 0
    for (owner, key), grad in cuda.items():
        a = grad.float().cpu().numpy().astype(np.float64).ravel()
        base = {"sc": sc, "av": av, "G": {"G": G}}[owner][key]
        flat_idx = rng.choice(base.size, size=min(base.size, 40), replace=False)
        kept, refs = central_differences(oracle, sc, av, G, cam, wr, wd, owner, key, flat_idx, h_rel=H_REL)
        assert len(refs) >= 20, (owner, key)
        check_grad(a[kept], refs, f"FD {path} {owner} {key}", 1e-3)
        checked += len(refs)
    assert checked > 300
