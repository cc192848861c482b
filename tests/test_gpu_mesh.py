"""The triangle-mesh layer on the GPU (gs_render_mesh) against the FP64
oracle, and the two-layer sensor of Sec. 3.2: a Gaussian scene composited
with a mesh by nearest depth."""
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


def compare_mesh(rgb, depth, ora):
    ok = ora["amb"] == 0
    d_rgb = np.abs(rgb.astype(np.float64) - ora["rgb"]).max(axis=0)
    d_dep = np.abs(depth.astype(np.float64) - ora["depth"]) / np.maximum(ora["depth"], 0.2)
    assert d_rgb[ok].max(initial=0.0) < 1e-4, d_rgb[ok].max()
    assert d_dep[ok].max(initial=0.0) < 1e-4, d_dep[ok].max()
    assert np.array_equal(depth[ok] > 0, ora["depth"][ok] > 0)
    assert ok.mean() > 0.95
    return float(1.0 - ok.mean())


def test_mesh_layer_matches_oracle_batched(gs, oracle):
    W, H = 120, 90  # not a multiple of the 16-pixel tile
    meshes = [synth.room_mesh(s, n_boxes=6 + 4 * s, grid=10) for s in range(3)]
    tri_off = np.cumsum([0] + [m["triangles"].shape[0] for m in meshes])
    v_off = np.cumsum([0] + [m["vertices"].shape[0] for m in meshes])
    cat = dict(vertices=np.concatenate([m["vertices"] for m in meshes]),
               colors=np.concatenate([m["colors"] for m in meshes]),
               triangles=np.concatenate([m["triangles"] + v_off[k] for k, m in enumerate(meshes)]))
    view_env = np.array([0, 1, 2, 1])  # env 1 seen by two views
    cams = np.stack([synth.room_camera(20 + v, W, H) for v in range(4)])
    rgb, depth = gs.render_mesh(gs.Mesh.from_numpy(cat), gs.Batch(tri_off, view_env), gs.cameras_tensor(cams), W, H,
                                bg=(0.1, 0.2, 0.3))
    torch.cuda.synchronize()
    for v, e in enumerate(view_env):
        m = meshes[e]
        ora = oracle.raster_mesh(m["vertices"], m["colors"], m["triangles"], cams[v], W, H, bg=(0.1, 0.2, 0.3))
        flagged = compare_mesh(rgb[v].cpu().numpy(), depth[v].cpu().numpy(), ora)
        print(f"view {v}: flagged {flagged:.4f}")


def test_gaussian_scene_composited_with_a_mesh(gs, oracle):
    """Sensor of a mixed scene: the Gaussian room (normalised depth) and a
    mesh layer merged per pixel by the nearer depth, against the same chain
    on the oracle's layers."""
    W = H = 96
    g = synth.room_scene(60_000, seed=31)
    mesh = synth.room_mesh(31, n_boxes=10)
    mesh["triangles"] = mesh["triangles"][6 * 2 * 64:]  # the boxes only: the Gaussian room is the background
    cam = synth.room_camera(31, W, H)
    ct = gs.cameras_tensor(cam[None])
    r = gs.Renderer(gs.Batch(np.array([0, g["means"].shape[0]])), W, H, normalize_depth=True)
    out = r.forward(gs.Gaussians.from_numpy(g), ct)
    mrgb, mdep = gs.render_mesh(gs.Mesh.from_numpy(mesh), gs.Batch(np.array([0, mesh["triangles"].shape[0]])), ct, W, H)
    rgb, dep = gs.composite_nearest(out[0], out[1], mrgb, mdep)
    torch.cuda.synchronize()
    om = oracle.raster_mesh(mesh["vertices"], mesh["colors"], mesh["triangles"], cam, W, H)
    compare_mesh(mrgb[0].cpu().numpy(), mdep[0].cpu().numpy(), om)
    assert (om["depth"] > 0).mean() > 0.05  # boxes in view
    sel_rgb, sel_dep = oracle.composite_nearest(out[0].cpu().numpy(), out[1].cpu().numpy(), mrgb.cpu().numpy(),
                                                mdep.cpu().numpy())
    np.testing.assert_array_equal(rgb.cpu().numpy(), sel_rgb.astype(np.float32))
    np.testing.assert_array_equal(dep.cpu().numpy(), sel_dep.astype(np.float32))
    gs_pix = (dep.cpu().numpy() == out[1].cpu().numpy()) & (out[1].cpu().numpy() > 0)
    assert 0.05 < gs_pix.mean() < 0.98  # both layers show
