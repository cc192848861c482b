"""gs_render_static -- the forward render for callers that cannot allocate
device memory (a plugin inside a host simulator whose device memory belongs to
another framework, or a path that must not allocate after start-up).  It keeps
its scratch in a 64 MiB array inside libgs, and gs_render_static_status reads
the device status word it leaves there.  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2604_12626_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def _outputs(V, H, W):
    return (torch.empty((V, 3, H, W), device="cuda"), torch.empty((V, H, W), device="cuda"),
            torch.empty((V, H, W), device="cuda"), torch.empty((V, H, W), dtype=torch.int32, device="cuda"))


def _call_static(api, G, batch, cams, cfg, out):
    # straight through the C ABI
    rgb, depth, T, nc = out
    st = api._lib.gs_render_static(ctypes.byref(G.c), ctypes.byref(batch.c), ctypes.c_void_p(cams.data_ptr()),
                                   ctypes.byref(cfg), ctypes.c_void_p(rgb.data_ptr()),
                                   ctypes.c_void_p(depth.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                   ctypes.c_void_p(nc.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def _static_status(api):
    v = ctypes.c_int32(123)
    st = api._lib.gs_render_static_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(v))
    assert st == 0
    return v.value


def test_static_scratch_matches_gs_render_on_two_calls_in_a_row(gs):
    W = H = 128
    cases = [(synth.room_scene(120_000, seed=61), synth.room_camera(61, W, H)),
             (synth.box_scene(5000, seed=62), synth.identity_camera(W, H))]
    for g, cam in cases:  # two calls in a row; the second must not see the first's leftovers
        n = g["means"].shape[0]
        batch = gs.Batch(np.array([0, n]))
        G = gs.Gaussians.from_numpy(g)
        ct = gs.cameras_tensor(cam[None])
        cfg = gs.make_config(W, H)
        assert gs.workspace_size(cfg, batch) <= gs.STATIC_SCRATCH_BYTES
        out_s = _outputs(1, H, W)
        assert _call_static(gs, G, batch, ct, cfg, out_s) == 0
        assert _static_status(gs) == 0
        ref = gs.Renderer(batch, W, H).forward(G, ct)  # the same configuration through gs_render
        torch.cuda.synchronize()
        for a, b, name in zip(out_s, ref, ("rgb", "depth", "T", "n_contrib")):
            assert torch.equal(a, b), name  # the same kernels on the same inputs: bit-identical
        assert (out_s[2] < 0.9).float().mean().item() > 0.05  # something was rendered


def test_static_call_allocates_no_device_memory(gs):
    W = H = 128
    g = synth.room_scene(100_000, seed=63)
    batch = gs.Batch(np.array([0, 100_000]))
    G = gs.Gaussians.from_numpy(g)
    ct = gs.cameras_tensor(synth.room_camera(63, W, H)[None])
    cfg = gs.make_config(W, H)
    out = _outputs(1, H, W)
    assert _call_static(gs, G, batch, ct, cfg, out) == 0  # set-up (and lazy module load) on the first call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call_static(gs, G, batch, ct, cfg, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_status_reports_capacity_overflow(gs):
    W = H = 128
    g = synth.box_scene(5000, seed=0)
    batch = gs.Batch(np.array([0, 5000]))
    G = gs.Gaussians.from_numpy(g)
    ct = gs.cameras_tensor(synth.identity_camera(W, H)[None])
    out = _outputs(1, H, W)
    assert _call_static(gs, G, batch, ct, gs.make_config(W, H, pair_capacity=1000), out) == 0
    assert _static_status(gs) == -4  # GS_ERR_CAPACITY
    assert _static_status(gs) == 0   # cleared by the read
    assert torch.isfinite(out[0]).all()
    assert _call_static(gs, G, batch, ct, gs.make_config(W, H), out) == 0
    assert _static_status(gs) == 0   # a call that fits reports nothing


def test_static_scratch_rejects_problems_beyond_its_size(gs):
    W = H = 256
    n = 2_000_000
    batch = gs.Batch(np.array([0, n]))
    cfg = gs.make_config(W, H)
    assert gs.workspace_size(cfg, batch) > gs.STATIC_SCRATCH_BYTES
    g = synth.box_scene(8, seed=0)
    G = gs.Gaussians.from_numpy(g)
    G.c.n = n  # only the sizes are checked before any work is enqueued
    out = _outputs(1, H, W)
    assert _call_static(gs, G, batch, gs.cameras_tensor(synth.identity_camera(W, H)[None]), cfg, out) == -3
