"""Forward parity of the CUDA path (through the C ABI) against the FP64 oracle,
bit-exact tile keys and order against a CPU reference, and the invariances the
definition implies (tile size, persistent grid, batching)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from helpers import compare_view, gpu_outputs, reference_keys  # noqa: E402
from paper_2604_12626_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def gs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_12626_gb300 import api

    return api


def render_gpu(api, g, cams, W, H, offs=None, view_env=None, sh_dtype=torch.float32, **kw):
    n = g["means"].shape[0]
    offs = np.array([0, n]) if offs is None else offs
    batch = api.Batch(offs, view_env)
    r = api.Renderer(batch, W, H, **kw)
    G = api.Gaussians.from_numpy(g, sh_dtype=sh_dtype)
    ct = api.cameras_tensor(cams)
    out = r.forward(G, ct)
    torch.cuda.synchronize()
    assert r.status() == 0
    return r, out, G, ct


def test_box_scene_matches_oracle_pixel_major(gs, oracle):
    g = synth.box_scene(5000, seed=0)
    W = H = 128
    cam = synth.identity_camera(W, H)
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H)
    ora = oracle.render(g, cam, W, H, mode="pixel")
    st = compare_view(gpu_outputs(out, 0), ora)
    print("box 5k 128x128:", st)
    stats = r.stats()
    assert stats["n_visible"] > 4000 and stats["n_pairs"] >= stats["n_visible"]


def _check_keys(r, cams, W, H, view_of_rec):
    s = r.sections()
    rec = s["records"].cpu().numpy()
    vis = s["vis"].cpu().numpy()
    bs = s["bin_start"].cpu().numpy().astype(np.int64)
    raw = s["keys"].cpu().numpy().view(np.uint64)[:bs[-1]]
    blended = (raw >> np.uint64(31)) & np.uint64(1)
    keys = raw & ~np.uint64(1 << 31)  # the blend flags pairs in bit 31 of the record word
    counts, ref = reference_keys(rec, vis, view_of_rec, cams, W, H, r.cfg.tile_w, r.cfg.tile_h)
    n_bins = s["n_bins"]
    assert np.array_equal(np.diff(bs), counts[:n_bins]), "bin counts (tile ranges) differ"
    assert np.array_equal(keys, ref), "sorted keys differ"
    quarters = s["quarters"].cpu().numpy().view(np.uint32)[:bs[-1]] if s["quarters"] is not None else None
    _check_blended_flags(rec, keys, blended.astype(bool), bs, cams, W, H, r.cfg.tile_w, r.cfg.tile_h, quarters)
    _check_window(rec, vis, view_of_rec, cams, W, H)
    return int(bs[-1])


def _check_window(rec, vis, view_of_rec, cams, W, H, sample=4000):
    """The pixel window (hx, hy) of a visible record holds every pixel where its
    alpha can reach 1/255: in FP64 from the record's own conic and opacity, on a
    sample of the records, every pixel of the image with power <= 0 and
    o e^power >= (1/255)(1 + 1e-4) lies inside the window; and the window is
    never wider than the square footprint r = ceil(3 sqrt(lambda_max)) of the
    2D covariance (the conic's inverse), up to the rounding of that inverse."""
    R = rec.shape[0]
    bits = np.unpackbits(vis.view(np.uint8), bitorder="little")[:R].astype(bool)
    idx = np.flatnonzero(bits)
    idx = np.random.default_rng(1).choice(idx, min(sample, idx.size), replace=False)
    r_ = rec[idx].astype(np.float64)
    uc, vc, hx, hy, A, B, C, op = (r_[:, k] for k in range(8))
    det = A * C - B * B
    a2, b2, c2 = C / det, -B / det, A / det  # the 2D covariance
    mid = 0.5 * (a2 + c2)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - a2 * c2 + b2 * b2))
    rad = np.ceil(3.0 * np.sqrt(lam) * (1 + 1e-6))
    assert np.all(hx <= rad) and np.all(hy <= rad), "window wider than the square footprint"
    v = view_of_rec[idx]
    ii = np.arange(W, dtype=np.float64)
    jj = np.arange(H, dtype=np.float64)
    for k in range(idx.size):
        dx = uc[k] - (ii - cams[v[k], 14])
        dy = vc[k] - (jj - cams[v[k], 15])
        nx = np.abs(dx) <= rad[k] + 1
        ny = np.abs(dy) <= rad[k] + 1
        if not nx.any() or not ny.any():
            continue
        DX, DY = np.meshgrid(dx[nx], dy[ny])
        power = -0.5 * (A[k] * DX * DX + C[k] * DY * DY) - B[k] * DX * DY
        reach = (power <= 0.0) & (op[k] * np.exp(np.minimum(power, 0.0)) >= (1.0 / 255.0) * (1.0 + 1e-4))
        reach &= (np.abs(DX) <= rad[k]) & (np.abs(DY) <= rad[k])
        outside = (np.abs(DX) > hx[k]) | (np.abs(DY) > hy[k])
        assert not np.any(reach & outside), ("window cuts a pixel that can blend", int(idx[k]))


def _check_blended_flags(rec, keys, blended, bs, cams, W, H, tw, th, quarters=None, sample=20000):
    """A pair flagged as blended has, at some pixel of its tile and inside its
    pixel window, power <= 0 and alpha >= 1/255 (checked in FP64 with a small
    margin on a sample of the flagged pairs).  With quarter bits (2 x 1 pixels
    per thread), a flagged pair names at least one quarter, and every 4 x 4
    quarter it names holds such a pixel."""
    assert blended.any(), "no pair flagged as blended"
    pos = np.flatnonzero(blended)
    pos = np.random.default_rng(0).choice(pos, min(sample, pos.size), replace=False)
    bins = np.searchsorted(bs, pos, side="right") - 1
    tiles_x, tiles_y = (W + tw - 1) // tw, (H + th - 1) // th
    v, t = bins // (tiles_x * tiles_y), bins % (tiles_x * tiles_y)
    ri = (keys[pos] & np.uint64(0x7FFFFFFF)).astype(np.int64)
    r_ = rec[ri].astype(np.float64)
    uc, vc, hx, hy, A, B, C, op = (r_[:, k] for k in range(8))
    ii = (t % tiles_x)[:, None] * tw + np.arange(tw)[None, :]
    jj = (t // tiles_x)[:, None] * th + np.arange(th)[None, :]
    dx = uc[:, None, None] - (ii[:, None, :] - cams[v, 14][:, None, None])
    dy = vc[:, None, None] - (jj[:, :, None] - cams[v, 15][:, None, None])
    inside = ((ii[:, None, :] < W) & (jj[:, :, None] < H) & (np.abs(dx) <= hx[:, None, None] + 1e-3)
              & (np.abs(dy) <= hy[:, None, None] + 1e-3))
    power = -0.5 * (A[:, None, None] * dx * dx + C[:, None, None] * dy * dy) - B[:, None, None] * dx * dy
    alpha = np.minimum(0.99, op[:, None, None] * np.exp(np.minimum(power, 0.0)))
    ok = inside & (power <= 1e-5) & (alpha >= (1.0 / 255.0) * (1.0 - 1e-4))
    assert ok.reshape(ok.shape[0], -1).any(axis=1).all(), "a pair flagged as blended reaches no pixel of its tile"
    if quarters is None:
        return
    qw = quarters[pos]
    assert np.all(qw != 0), "a pair flagged as blended names no quarter"
    # ok[k, y, x] over the tile's pixels; quarter (w, q) covers block rows/cols
    nbx = tw // 8
    for w_ in range(nbx * (th // 8)):
        for q in range(4):
            sel = ((qw >> np.uint32(8 * w_ + q)) & np.uint32(1)).astype(bool)
            if not sel.any():
                continue
            y0 = (w_ // nbx) * 8 + (q >> 1) * 4
            x0 = (w_ % nbx) * 8 + (q & 1) * 4
            blk = ok[sel][:, y0:y0 + 4, x0:x0 + 4].reshape(int(sel.sum()), -1)
            assert blk.any(axis=1).all(), ("a quarter flagged as blended holds no pixel that can blend", w_, q)


def test_box_scene_keys_bit_exact(gs):
    g = synth.box_scene(5000, seed=0)
    W = H = 128
    cam = synth.identity_camera(W, H)
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H)
    P = _check_keys(r, cam[None], W, H, np.zeros(5000, np.int64))
    assert P > 5000


@pytest.fixture(scope="module")
def room1m():
    g = synth.room_scene(1_000_000, seed=1)
    cam = synth.room_camera(1, 640, 480)
    return g, cam


def test_room_1m_640x480_matches_oracle(gs, oracle, room1m):
    g, cam = room1m
    W, H = 640, 480
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H)
    ora = oracle.render(g, cam, W, H)
    st = compare_view(gpu_outputs(out, 0), ora)
    print("room 1M 640x480:", st, r.stats())


def test_room_1m_keys_bit_exact(gs, room1m):
    g, cam = room1m
    W, H = 640, 480
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H)
    P = _check_keys(r, cam[None], W, H, np.zeros(g["means"].shape[0], np.int64))
    assert P > 100_000


@pytest.mark.parametrize("tile,depth", [((8, 8), 64), ((16, 16), 128), ((16, 8), 36)])
def test_quarter_lists_keys_and_flags(gs, tile, depth):
    """2 x 1 pixels per thread (a Gaussian list per 4 x 4 quarter): keys and
    tile ranges bit-exact, the blended flags and the quarter bits reach pixels
    that can blend, and the images equal the one-pixel-per-thread path."""
    g = synth.room_scene(300_000, seed=8)
    W = H = 256
    cam = synth.room_camera(8, W, H)
    r, b, _, _ = render_gpu(gs, g, cam[None], W, H, tile=tile, batch_depth=depth, pix=(2, 1), persistent=True)
    _check_keys(r, cam[None], W, H, np.zeros(g["means"].shape[0], np.int64))
    _, a, _, _ = render_gpu(gs, g, cam[None], W, H, tile=tile, pix=(1, 1))
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("tile,depth,pix", [((8, 8), 64, (1, 1)), ((16, 8), 128, (1, 1)), ((32, 8), 256, (1, 1)),
                                            ((32, 16), 32, (1, 1)), ((16, 16), 256, (2, 2)), ((8, 8), 128, (2, 1)),
                                            ((16, 8), 64, (1, 2)), ((16, 16), 128, (2, 1)),
                                            ((8, 8), 36, (2, 1)), ((16, 8), 100, (1, 1))])
def test_tile_size_does_not_change_results(gs, tile, depth, pix):
    # (batch depths 36 and 100: not multiples of the blend loop's 8 Gaussians)
    g = synth.room_scene(200_000, seed=4)
    W, H = 200, 150  # not a multiple of any tile
    cam = synth.room_camera(4, W, H)
    _, a, _, _ = render_gpu(gs, g, cam[None], W, H)
    _, b, _, _ = render_gpu(gs, g, cam[None], W, H, tile=tile, batch_depth=depth, pix=pix)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("pix", [(1, 1), (2, 2)])
def test_persistent_grid_equals_one_cta_per_tile(gs, pix):
    g = synth.room_scene(300_000, seed=5)
    W = H = 256
    cam = synth.room_camera(5, W, H)
    _, a, _, _ = render_gpu(gs, g, cam[None], W, H)
    _, b, _, _ = render_gpu(gs, g, cam[None], W, H, persistent=True, pix=pix)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.fixture(scope="module")
def small_batch():
    return synth.batched_rooms(n_envs=6, n_min=30_000, n_max=150_000, W=256, H=256, seed0=100)


def test_batched_equals_per_env_loop(gs, small_batch):
    g, offs, cams = small_batch
    W = H = 256
    _, ab, _, _ = render_gpu(gs, g, cams, W, H, offs=offs, persistent=True)
    for e in range(len(offs) - 1):
        ge = {k: v[offs[e]:offs[e + 1]] for k, v in g.items()}
        _, ae, _, _ = render_gpu(gs, ge, cams[e:e + 1], W, H)
        for x, y in zip(ab, ae):
            assert torch.equal(x[e], y[0])


def test_batched_matches_oracle(gs, oracle, small_batch):
    g, offs, cams = small_batch
    W = H = 256
    r, out, _, _ = render_gpu(gs, g, cams, W, H, offs=offs, persistent=True)
    for e in range(len(offs) - 1):
        ge = {k: v[offs[e]:offs[e + 1]] for k, v in g.items()}
        compare_view(gpu_outputs(out, e), oracle.render(ge, cams[e], W, H))
    views = np.repeat(np.arange(len(offs) - 1), np.diff(offs))
    _check_keys(r, cams, W, H, views)


def test_views_sharing_an_env(gs, oracle):
    # several cameras on one scene: one record per (view, Gaussian)
    g = synth.room_scene(150_000, seed=7)
    W = H = 128
    cams = np.stack([synth.room_camera(20 + k, W, H) for k in range(4)])
    r, out, _, _ = render_gpu(gs, g, cams, W, H, offs=np.array([0, 150_000]), view_env=[0, 0, 0, 0])
    for v in range(4):
        compare_view(gpu_outputs(out, v), oracle.render(g, cams[v], W, H))
    _check_keys(r, cams, W, H, np.repeat(np.arange(4), 150_000))


@pytest.mark.parametrize("dt", ["f16", "bf16"])
def test_half_precision_sh_storage(gs, oracle, dt):
    g = synth.room_scene(200_000, seed=8)
    W = H = 256
    cam = synth.room_camera(8, W, H)
    tdt = torch.float16 if dt == "f16" else torch.bfloat16
    _, out, _, _ = render_gpu(gs, g, cam[None], W, H, sh_dtype=tdt)
    gq = dict(g)
    if dt == "f16":
        gq["sh"] = g["sh"].astype(np.float16).astype(np.float32)
    else:
        gq["sh"] = synth.bf16_to_f32(synth.bf16_bits(g["sh"]))
    st = compare_view(gpu_outputs(out, 0), oracle.render(gq, cam, W, H))  # exact on the stored values
    full = oracle.render(g, cam, W, H)
    err = np.abs(out[0][0].cpu().numpy() - full["rgb"]).max()
    print(f"SH {dt}: vs quantised-input oracle {st}, vs FP32-input oracle max |rgb| err {err:.2e}")
    assert err < (2e-3 if dt == "f16" else 2e-2)


def test_background_and_normalised_depth(gs, oracle):
    g = synth.box_scene(3000, seed=9)
    W = H = 64
    cam = synth.identity_camera(W, H)
    bg = (0.2, 0.5, 0.9)
    _, out, _, _ = render_gpu(gs, g, cam[None], W, H, bg=bg, normalize_depth=True)
    compare_view(gpu_outputs(out, 0), oracle.render(g, cam, W, H, bg=bg, normalize_depth=True))


def test_edge_cases(gs, oracle):
    W, H = 37, 23
    cam = synth.identity_camera(W, H)
    # everything behind the camera or beyond the near plane
    g = synth.box_scene(500, seed=10)
    g["means"][:, 2] = np.float32(-1.0)
    _, out, _, _ = render_gpu(gs, g, cam[None], W, H)
    assert torch.all(out[2] == 1.0) and torch.all(out[0] == 0.0) and torch.all(out[3] == 0)
    # an empty env next to a non-empty one; 1x1 image
    g = synth.box_scene(400, seed=11)
    g["log_scales"] += np.float32(2.0)
    offs = np.array([0, 0, 400])
    c1 = synth.identity_camera(1, 1)
    r, out, _, _ = render_gpu(gs, g, np.stack([c1, c1]), 1, 1, offs=offs)
    assert torch.all(out[2][0] == 1.0)
    compare_view(gpu_outputs(out, 1), oracle.render(g, c1, 1, 1))
    # one Gaussian covering the whole image
    g = dict(means=np.float32([[0.0, 0.0, 3.0]]), log_scales=np.float32([[1.0, 1.0, 1.0]]),
             quats=np.float32([[1, 0, 0, 0]]), opacity_logits=np.float32([2.0]), sh=np.zeros((1, 16, 3), np.float32))
    _, out, _, _ = render_gpu(gs, g, cam[None], W, H)
    compare_view(gpu_outputs(out, 0), oracle.render(g, cam, W, H))


def test_capacity_overflow_is_reported_not_written(gs):
    g = synth.box_scene(5000, seed=0)
    W = H = 128
    cam = synth.identity_camera(W, H)
    batch = gs.Batch(np.array([0, 5000]))
    r = gs.Renderer(batch, W, H, pair_capacity=1000)
    G = gs.Gaussians.from_numpy(g)
    out = r.forward(G, gs.cameras_tensor(cam[None]))
    torch.cuda.synchronize()
    assert r.status() == -4  # GS_ERR_CAPACITY
    assert r.status() == 0   # cleared by the read
    assert torch.isfinite(out[0]).all()


@pytest.mark.parametrize("tile,persistent", [((16, 16), False), ((8, 8), True)])
def test_evaluation_count_matches_oracle(gs, oracle, tile, persistent):
    """GS_FLAG_COUNT_EVALS: per pixel, the covered Gaussians examined in depth
    order up to and including the one that stops it, summed -- the oracle's own
    count.  Scene and seed are chosen so that the oracle flags no pixel whose
    count FP32 rounding could change, so the two must agree exactly."""
    g = synth.box_scene(1500, seed=2)
    g["opacity_logits"] = g["opacity_logits"] + 3.0  # opaque enough that pixels stop
    W = H = 64
    cam = synth.identity_camera(W, H)
    ora = oracle.render(g, cam, W, H, mode="gaussian")
    assert not np.any(ora["amb"] & 2)
    r, out, G, ct = render_gpu(gs, g, cam[None], W, H, tile=tile, persistent=persistent)
    assert r.stats()["n_evaluations"] == 0  # not counted without the flag
    ev = r.count_evaluations(G, ct)
    assert ev == ora["evals"], (ev, ora["evals"])
    assert ev > int(ora["n_contrib"].sum())  # skipped and stopping Gaussians are counted too
    # the adjoint's walk: covered Gaussians up to each pixel's last blended one
    assert r.stats()["n_covered"] == int(ora["n_covered"].sum())
    assert int(ora["n_covered"].sum()) > int(ora["n_contrib"].sum())


def test_large_bins_keys_bit_exact(gs):
    """Bins of tens of thousands of pairs: 4096-key chunk sorts, then several
    merge passes (runs of 4096, 8192, ...) that must end in the keys buffer."""
    g = synth.room_scene(400_000, seed=7)
    W = H = 64
    cam = synth.room_camera(7, W, H)
    with pytest.raises(gs.GsError, match="UNSUPPORTED"):  # 1024 threads: more registers than an SM has
        render_gpu(gs, g, cam[None], W, H, tile=(32, 32), batch_depth=256)
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H, tile=(32, 32), batch_depth=256, pix=(2, 2))
    assert r.stats()["max_bin"] > 4 * 4096
    _check_keys(r, cam[None], W, H, np.zeros(g["means"].shape[0], np.int64))


@pytest.mark.parametrize("n", [3000, 9000])
def test_wide_depth_range_keys_bit_exact(gs, n):
    """Depths from 0.3 m to 100 km inside the same tiles: their FP32 bit patterns
    span more than 2^27, so the bin sort takes its four 8-bit passes over the
    depth bits instead of three 9-bit passes over the offset depths."""
    rng = np.random.default_rng(n)
    z = np.exp(rng.uniform(np.log(0.3), np.log(1e5), n))
    xy = rng.uniform(-0.02, 0.02, (n, 2)) * z[:, None]  # within a few pixels of the axis
    g = synth.box_scene(n, seed=n)
    g["means"] = np.stack([xy[:, 0], xy[:, 1], z], 1).astype(np.float32)
    g["log_scales"] = np.log(0.01 * z)[:, None].repeat(3, 1).astype(np.float32)  # about a pixel at any depth
    W = H = 64
    cam = synth.identity_camera(W, H)
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H, tile=(8, 8), batch_depth=64)
    zk = np.sort(g["means"][:, 2])
    assert zk.view(np.uint32)[-1] - zk.view(np.uint32)[0] > (1 << 27)
    assert r.stats()["max_bin"] > 2048
    _check_keys(r, cam[None], W, H, np.zeros(n, np.int64))


@pytest.mark.parametrize("n", [3000, 20_000])
def test_equal_depths_sorted_by_record_index(gs, oracle, n):
    """Every Gaussian at exactly the same FP32 depth: the order inside a bin is
    then the record index alone (within one chunk and across merged chunks)."""
    rng = np.random.default_rng(11)
    g = dict(means=np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.8, 0.8, n), np.full(n, 3.0)], 1).astype(np.float32),
             log_scales=rng.normal(-3.0, 0.3, (n, 3)).astype(np.float32),
             quats=rng.normal(size=(n, 4)).astype(np.float32),
             opacity_logits=rng.normal(0, 1, n).astype(np.float32),
             sh=(rng.normal(0, 0.1, (n, 16, 3))).astype(np.float32))
    W = H = 32
    cam = synth.identity_camera(W, H)
    r, out, _, _ = render_gpu(gs, g, cam[None], W, H, tile=(16, 16))
    _check_keys(r, cam[None], W, H, np.zeros(n, np.int64))
    if n > 4096:
        assert r.stats()["max_bin"] > 4096
    compare_view(gpu_outputs(out, 0), oracle.render(g, cam, W, H))
