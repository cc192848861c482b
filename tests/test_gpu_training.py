"""The forward + backward training workload at full size: one 500k-Gaussian
room plus two 50k-Gaussian avatars (24 joints) posed by LBS, 16 views at
512x512, an L1 loss against a target rendered from perturbed parameters
(means + N(0, 1 cm), SH + N(0, 0.02)), through api.AvatarScene -- the
preallocated step the benchmark times (gs_deform_avatars, gs_render,
gs_render_backward in overwrite mode, gs_deform_avatars_backward).  Two views'
images against the FP64 oracle; the gradients of every scene and avatar
parameter and of the joint transforms, summed over all 16 views, against the
oracle's adjoint (LBS in FP64, posed rows flagged inexact), per group by
relative L2 and element by element.  FP32 and FP16 SH storage, and the fused
path (gs_render_avatars, gs_render_avatars_backward: the avatars posed inside
the render).  Paper:
differentiable rasterisation (Sec. 2.2, Sec. 3.2) of scenes with avatars
(Sec. 3.3)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_grad, compare_view, gpu_outputs  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402

W = H = 512
V = 16
KW = dict(tile=(16, 16), batch_depth=128, pix=(2, 1), persistent=True)


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


@pytest.fixture(scope="module")
def workload():
    return synth.training_scene(seed=0, W=W, H=H, n_views=V)


def _scene(gs, wl, sh_dtype, perturbed=False, fused=False):
    T = lambda x, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)  # noqa: E731
    room, av = wl["room"], wl["avatars"]
    rm, rsh, am, ash = room["means"], room["sh"], av["means"], av["sh"]
    if perturbed:
        rm, rsh, am, ash = rm + wl["d_room_means"], rsh + wl["d_room_sh"], am + wl["d_av_means"], ash + wl["d_av_sh"]
    scene = dict(means=T(rm), log_scales=T(room["log_scales"]), quats=T(room["quats"]),
                 opacity_logits=T(room["opacity_logits"]), sh=T(rsh))
    avatars = dict(means=T(am), log_scales=T(av["log_scales"]), quats=T(av["quats"]),
                   opacity_logits=T(av["opacity_logits"]), sh=T(ash), joint_ids=T(av["joint_ids"].view(np.int16),
                                                                                   torch.int16),
                   weights=T(av["weights"]), avatar_of=T(av["avatar_of"], torch.int32))
    return gs.AvatarScene(scene, avatars, wl["G"].shape[0], 24, W, H, V, sh_dtype=sh_dtype, fused=fused, **KW)


@pytest.mark.parametrize("sh_dtype,fused", [(torch.float32, False), (torch.float16, False), (torch.float32, True)],
                         ids=["f32", "f16", "f32-fused"])
def test_training_step_matches_oracle(gs, oracle, workload, sh_dtype, fused):
    wl = workload
    cams = gs.cameras_tensor(wl["cams"])
    G = torch.from_numpy(wl["G"]).cuda()
    tgt = _scene(gs, wl, sh_dtype, perturbed=True)
    t_rgb, t_depth = (x.clone() for x in tgt.forward(G, cams)[:2])
    del tgt
    sc = _scene(gs, wl, sh_dtype, fused=fused)
    out = sc.forward(G, cams)
    d_rgb = torch.sign(out[0] - t_rgb)
    d_depth = 0.1 * torch.sign(out[1] - t_depth)
    torch.cuda.synchronize()
    assert sc.renderer.status() == 0
    assert float((out[0] - t_rgb).abs().mean()) > 1e-3  # the perturbed target differs

    # the oracle's input: FP64 LBS of the canonical avatars, posed rows by covariance
    room, av = wl["room"], wl["avatars"]
    q = (lambda x: x.astype(np.float16).astype(np.float32)) if sh_dtype == torch.float16 else (lambda x: x)
    pm, pc = oracle.lbs(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32), av["weights"],
                        av["avatar_of"], wl["G"].astype(np.float64))
    ns, m = room["means"].shape[0], av["means"].shape[0]
    g = dict(means=np.concatenate([room["means"].astype(np.float64), pm]),
             log_scales=np.concatenate([room["log_scales"], np.zeros((m, 3), np.float32)]),
             quats=np.concatenate([room["quats"], np.tile(np.float32([1, 0, 0, 0]), (m, 1))]),
             opacity_logits=np.concatenate([room["opacity_logits"], av["opacity_logits"]]),
             sh=q(np.concatenate([room["sh"], av["sh"]])), cov3d=np.concatenate([np.zeros((ns, 6)), pc]),
             use_cov=np.concatenate([np.zeros(ns, np.uint8), np.ones(m, np.uint8)]),
             inexact=np.concatenate([np.zeros(ns, np.uint8), np.ones(m, np.uint8)]))
    up_rgb = d_rgb.cpu().numpy().astype(np.float64)
    up_depth = d_depth.cpu().numpy().astype(np.float64)
    for v in range(V):
        ora = oracle.render(g, wl["cams"][v], W, H)
        if v < 2:  # views 0 and 1 each have an avatar 2 m in front of the camera
            compare_view(gpu_outputs(out, v), ora)
        amb = ora["amb"] != 0
        up_rgb[v][:, amb] = 0.0
        up_depth[v][amb] = 0.0
    grads, av_grads = sc.backward(G, cams, torch.from_numpy(up_rgb).float().cuda(),
                                  torch.from_numpy(up_depth).float().cuda())
    torch.cuda.synchronize()
    assert sc.renderer.status() == 0

    def view_grads(v):  # the oracle releases the GIL: views run side by side in threads
        return oracle.render_backward(g, wl["cams"][v], W, H, up_rgb[v], up_depth[v])

    with ThreadPoolExecutor(max_workers=8) as ex:
        per_view = list(ex.map(view_grads, range(V)))
    og = {k: sum(p[k] for p in per_view) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "cov3d")}
    oga = oracle.lbs_backward(av["means"], av["log_scales"], av["quats"], av["joint_ids"].astype(np.int32),
                              av["weights"], av["avatar_of"], wl["G"].astype(np.float64), og["means"][ns:],
                              og["cov3d"][ns:])
    gg = {k: v.cpu().numpy() for k, v in grads.items()}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        check_grad(gg[k][:ns], og[k][:ns], f"room {k}", 1e-3)
    for k in ("opacity_logits", "sh"):
        check_grad(gg[k][ns:], og[k][ns:], f"avatar {k}", 1e-3)
    for k in ("means", "log_scales", "quats", "G"):
        check_grad(av_grads[k].cpu().numpy(), oga[k], f"avatar canonical {k}", 1e-3)
    assert np.abs(oga["G"]).max() > 0  # the joints are seen
