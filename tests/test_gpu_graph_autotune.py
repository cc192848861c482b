"""The batched form (a11): gs_render + gs_render_backward of a multi-env batch
captured in one CUDA graph and replayed with new cameras, against eager calls
and the FP64 oracle; and gs_autotune, the tile / batch-depth / pixels-per-thread
tuner the batched renderer is launched with.  The paper renders one env per
call (Table 6, Sec. 4.5); this batching is the GB300 addition it is compared
with."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import check_grad, compare_view, gpu_outputs  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")
W = H = 128
KW = dict(tile=(8, 8), batch_depth=64, pix=(2, 1), persistent=True, grad_overwrite=True)


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def _grads(n, dev="cuda"):
    return dict(means=torch.empty((n, 3), device=dev), log_scales=torch.empty((n, 3), device=dev),
                quats=torch.empty((n, 4), device=dev), opacity_logits=torch.empty((n,), device=dev),
                sh=torch.empty((n, 16, 3), device=dev))


def test_graph_replay_with_new_cameras_equals_eager_and_oracle(gs, oracle):
    g, offs, cams0 = synth.batched_rooms(4, 30_000, 90_000, W, H, seed0=500)
    n = int(offs[-1])
    G = gs.Gaussians.from_numpy(g, sh_dtype=torch.float16)
    batch = gs.Batch(offs)
    rng = np.random.default_rng(8)
    d_rgb = torch.from_numpy(rng.standard_normal((4, 3, H, W)).astype(np.float32)).cuda()
    d_depth = torch.from_numpy((0.1 * rng.standard_normal((4, H, W))).astype(np.float32)).cuda()
    # the graph's static inputs and outputs
    rend = gs.Renderer(batch, W, H, **KW)
    cams_dev = gs.cameras_tensor(cams0)
    outs = rend.alloc_outputs()
    grads = _grads(n)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # one eager step first (as before any capture)
        rend.forward(G, cams_dev, out=outs, stream=s)
        rend.backward(G, cams_dev, d_rgb, d_depth, grads=grads, stream=s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rend.forward(G, cams_dev, out=outs, stream=s)
        rend.backward(G, cams_dev, d_rgb, d_depth, grads=grads, stream=s)
    eager = gs.Renderer(batch, W, H, **KW)
    for rep, seed in enumerate((700, 800)):  # two replays, each with new cameras copied in
        cams = np.stack([synth.room_camera(seed + e, W, H) for e in range(4)])
        cams_dev.copy_(gs.cameras_tensor(cams))
        graph.replay()
        torch.cuda.synchronize()
        assert rend.status() == 0
        ct = gs.cameras_tensor(cams)
        ref = eager.forward(G, ct)
        ref_g = eager.backward(G, ct, d_rgb, d_depth, grads=_grads(n))
        torch.cuda.synchronize()
        for a, b, name in zip(outs, ref, ("rgb", "depth", "T", "n_contrib")):
            assert torch.equal(a, b), (rep, name)  # the forward is deterministic: bit-identical
        for k in GROUPS:  # float atomics in tile-completion order: equal up to rounding (a stale row
            # or a doubled gradient would be off by the gradient itself)
            check_grad(grads[k].cpu().numpy(), ref_g[k].cpu().numpy(), f"replay {rep} {k}", 2e-5)
        sh16 = g["sh"].astype(np.float16).astype(np.float32)
        for e in range(4):
            sl = slice(int(offs[e]), int(offs[e + 1]))
            ge = {k: np.asarray(v[sl]) for k, v in g.items()}
            ge["sh"] = sh16[sl]
            compare_view(gpu_outputs(outs, e), oracle.render(ge, cams[e], W, H))
        assert (outs[2] < 0.5).float().mean().item() > 0.2  # the rooms are rendered, not empty


CANDIDATES = [(16, 16, 256, 1, 1), (16, 16, 128, 2, 2), (16, 8, 128, 2, 1), (8, 8, 64, 2, 1), (8, 8, 64, 1, 1),
              (32, 16, 256, 2, 2)]


def test_autotune_returns_a_candidate_and_results_do_not_depend_on_it(gs):
    g, offs, cams = synth.batched_rooms(3, 30_000, 90_000, W, H, seed0=600)
    G = gs.Gaussians.from_numpy(g, sh_dtype=torch.float16)
    batch = gs.Batch(offs)
    ct = gs.cameras_tensor(cams)
    fixed = gs.Renderer(batch, W, H, tile=(16, 16), batch_depth=256)
    ref = [t.clone() for t in fixed.forward(G, ct)]
    r = gs.Renderer(batch, W, H, persistent=True, tile_candidates=CANDIDATES)
    choice, best_ms = r.autotune(G, ct, CANDIDATES, reps=2)
    assert tuple(choice) in CANDIDATES and best_ms > 0.0
    out = r.forward(G, ct)
    torch.cuda.synchronize()
    assert r.status() == 0
    for a, b, name in zip(out, ref, ("rgb", "depth", "T", "n_contrib")):
        assert torch.equal(a, b), (choice, name)  # the footprint is per pixel: no tile dependence


def test_autotune_skips_candidates_that_do_not_fit_the_workspace(gs):
    g, offs, cams = synth.batched_rooms(2, 30_000, 60_000, W, H, seed0=650)
    G = gs.Gaussians.from_numpy(g)
    batch = gs.Batch(offs)
    ct = gs.cameras_tensor(cams)
    small = (8, 8, 64, 2, 1)
    r = gs.Renderer(batch, W, H, tile=small[:2], batch_depth=small[2], pix=small[3:])  # sized for `small` only
    big = [c for c in CANDIDATES if gs.workspace_size(
        gs.make_config(W, H, tile=c[:2], batch_depth=c[2], pix=c[3:]), batch) > r.ws_bytes]
    assert len(big) >= 2
    choice, _ = r.autotune(G, ct, big + [small], reps=1)
    assert tuple(choice) == small  # every larger candidate was skipped, not run out of bounds
    ref = gs.Renderer(batch, W, H).forward(G, ct)
    out = r.forward(G, ct)
    torch.cuda.synchronize()
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    with pytest.raises(gs.GsError, match="WORKSPACE_TOO_SMALL"):
        r.autotune(G, ct, big, reps=1)  # nothing fits
