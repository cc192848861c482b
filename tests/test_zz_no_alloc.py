"""gs_render_static -- the forward render for callers that cannot allocate
device memory (a plugin inside a host simulator whose device memory belongs to
another framework, or a path that must not allocate after start-up).  It keeps
its scratch in a 64 MiB array inside libgs.  This file is collected last so
that a run stopping at the first failure has already run every other test."""
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
        ref = gs.Renderer(batch, W, H).forward(G, ct)
        torch.cuda.synchronize()
        rgb_s, dep_s, T_s, nc_s = (t.cpu().numpy() for t in out_s)
        rgb_r, dep_r, T_r, nc_r = (t.cpu().numpy() for t in ref)
        assert np.abs(rgb_s - rgb_r).max() <= 1e-4
        assert (np.abs(dep_s - dep_r) / np.maximum(dep_r, 0.2)).max() <= 1e-4
        assert np.abs(T_s - T_r).max() <= 1e-4
        assert np.array_equal(nc_s, nc_r)
        assert (T_s < 0.9).mean() > 0.05  # something was rendered


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
