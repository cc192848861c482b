"""The precision form: SH coefficients stored as FP32, FP16 or BF16, with
projection, conic and blending in FP32, each output compared with the FP64
oracle run on the original FP32 inputs (so the error includes the storage
rounding of the coefficients).  Per form: the largest colour, depth and
transmittance errors over the pixels the oracle does not flag, and the
relative L2 error of every parameter-gradient group against the oracle
adjoint (upstream gradient zero at flagged pixels).  The figures are printed,
written as JSON where GS_PRECISION_OUT names a file, and bounded here."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import DEPTH_FLOOR, rel_l2  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402
from test_gpu_backward import GROUPS, gpu_forward_backward, mask_ambiguous, oracle_grads  # noqa: E402

# bounds on the errors against the FP32-input oracle: FP32 storage keeps the
# 1e-4 image tolerance; the 16-bit forms add the rounding of the coefficients
# (relative 2^-11 for FP16, 2^-8 for BF16) times the colour they make
RGB_MAX = {"f32": 1e-4, "f16": 2e-3, "bf16": 2e-2}
GRAD_L2 = {"f32": 1e-3, "f16": 1e-2, "bf16": 5e-2}


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


@pytest.fixture(scope="module")
def scene(oracle):
    g = synth.room_scene(200_000, seed=8)
    W = H = 256
    cam = synth.room_camera(8, W, H)
    ora = oracle.render(g, cam, W, H)
    rng = np.random.default_rng(8)
    d_rgb = rng.standard_normal((1, 3, H, W)).astype(np.float32)
    d_depth = rng.standard_normal((1, H, W)).astype(np.float32)
    mask_ambiguous(oracle, g, cam[None], W, H, d_rgb, d_depth)
    og = oracle_grads(oracle, g, cam[None], W, H, d_rgb, d_depth)
    return g, cam, W, H, ora, d_rgb, d_depth, og


_RESULTS = {}


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_error_of_each_output_per_storage_type(gs, scene, dt):
    g, cam, W, H, ora, d_rgb, d_depth, og = scene
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dt]
    r = gs.Renderer(gs.Batch(np.array([0, g["means"].shape[0]])), W, H, tile=(16, 8), batch_depth=128, pix=(2, 1),
                    persistent=True)
    G = gs.Gaussians.from_numpy(g, sh_dtype=tdt)
    ct = gs.cameras_tensor(cam[None])
    rgb, depth, T, _ = (x.cpu().numpy()[0] for x in r.forward(G, ct))
    ok = (ora["amb"] & 1) == 0
    st = dict(
        rgb_max=float(np.abs(rgb - ora["rgb"]).max(axis=0)[ok].max()),
        rgb_p999=float(np.quantile(np.abs(rgb - ora["rgb"]).max(axis=0)[ok], 0.999)),
        depth_rel_max=float((np.abs(depth - ora["depth"]) / np.maximum(ora["depth"], DEPTH_FLOOR))[ok].max()),
        T_max=float(np.abs(T - ora["T"])[ok].max()),
        flagged_frac=float((~ok).mean()),
    )
    a = gpu_forward_backward(gs, g, cam[None], W, H, d_rgb, d_depth, sh_dtype=tdt, tile=(16, 8), batch_depth=128,
                             pix=(2, 1), persistent=True)
    for k in GROUPS:
        st[f"grad_{k}_rel_l2"] = rel_l2(a[k], og[k])
    _RESULTS[dt] = st
    print(f"SH stored {dt}:", json.dumps(st))
    out = os.environ.get("GS_PRECISION_OUT")
    if out:
        with open(out, "w") as f:
            json.dump({"scene": "room 200k Gaussians, 256x256, seed 8; oracle on the FP32 inputs",
                       "forms": _RESULTS}, f, indent=1)
    assert st["rgb_max"] <= RGB_MAX[dt], st
    assert st["T_max"] <= 1e-4, st  # transmittance does not depend on the colour
    assert st["depth_rel_max"] <= 1e-4, st  # neither does depth
    for k in GROUPS:
        assert st[f"grad_{k}_rel_l2"] <= GRAD_L2[dt], (k, st)
