"""Shared helpers of the GPU tests: oracle comparison with the ambiguous-pixel
mask, and an independent CPU reference for the integer stages (tile binning
and key order) computed from the GPU's own projected records."""
from __future__ import annotations

import numpy as np

AMB_VALUE, AMB_COUNT = 1, 2
TOL_RGB = 1e-4          # max-abs per channel, FP32 vs FP64
TOL_DEPTH_REL = 1e-4    # relative to the oracle depth
DEPTH_FLOOR = 0.2       # near plane: depth tolerance floor is 1e-4 * 0.2
MAX_BAD = 1e-4          # fraction of pixels allowed beyond tolerance (all must be flagged)
MAX_FLAGGED = 0.05      # sanity bound on the oracle's ambiguous fraction
# FP32 rounding accumulated over a pixel's blend (amplified by alpha / (1 - alpha)
# for near-opaque contributors) can carry a value past the tolerance with no
# decision near its threshold; such a pixel must keep the oracle's contributor
# count and stay within this multiple of the tolerance
CONT_FACTOR = 2.0


def compare_view(gpu: dict, ora: dict, tol_rgb=TOL_RGB, tol_depth=TOL_DEPTH_REL):
    """gpu: rgb [3,H,W], depth, T, n_contrib (numpy); ora: oracle.render output.

    A pixel is out of tolerance if any channel differs by more than 1e-4 or the
    depth by more than 1e-4 x max(depth, 0.2).  FP32 rounding can flip a discrete
    decision (footprint, alpha >= 1/255, T < 1e-4) only where the oracle flags
    the pixel as ambiguous, so: every out-of-tolerance pixel must be flagged or
    be a rounding excess (the oracle's contributor count, within CONT_FACTOR x
    the tolerance), at most ceil(1e-4 x pixels) may be out of tolerance, and
    contributor counts must agree wherever no count-changing decision was
    flagged."""
    amb_v = (ora["amb"] & AMB_VALUE) != 0
    amb_c = (ora["amb"] & AMB_COUNT) != 0
    d_rgb = np.abs(gpu["rgb"].astype(np.float64) - ora["rgb"]).max(axis=0)
    d_dep = np.abs(gpu["depth"].astype(np.float64) - ora["depth"])
    d_rel = d_dep / np.maximum(ora["depth"], DEPTH_FLOOR)
    d_T = np.abs(gpu["T"].astype(np.float64) - ora["T"])
    bad = (d_rgb > tol_rgb) | (d_rel > tol_depth) | (d_T > tol_rgb)
    near = (d_rgb <= CONT_FACTOR * tol_rgb) & (d_rel <= CONT_FACTOR * tol_depth) & (d_T <= CONT_FACTOR * tol_rgb)
    rounding = bad & ~amb_v & near & (gpu["n_contrib"] == ora["n_contrib"])
    ok = ~amb_v
    st = dict(
        max_rgb=float(d_rgb[ok].max(initial=0.0)),
        max_depth_rel=float(d_rel[ok].max(initial=0.0)),
        max_T=float(d_T[ok].max(initial=0.0)),
        bad=int(bad.sum()),
        bad_frac=float(bad.mean()),
        amb_frac=float(amb_v.mean()),
        count_mismatch=int(((gpu["n_contrib"] != ora["n_contrib"]) & ~amb_c).sum()),
        rounding=int(rounding.sum()),
    )
    assert not np.any(bad & ~amb_v & ~rounding), st
    assert st["bad"] <= max(1, int(np.ceil(MAX_BAD * bad.size))), st
    assert st["amb_frac"] <= MAX_FLAGGED, st
    assert st["count_mismatch"] == 0, st
    return st


def covered_range(u_c: np.float32, r: np.float32, c: np.float32, n: int):
    """First/last pixel index in [0, n) with |u_c - (i - c)| <= r evaluated in
    FP32 -- brute force over all pixels (the definition of the footprint)."""
    pix = np.arange(n, dtype=np.float32) - np.float32(c)
    cov = np.abs(np.float32(u_c) - pix) <= np.float32(r)
    idx = np.flatnonzero(cov)
    if idx.size == 0:
        return None
    return int(idx[0]), int(idx[-1])


def covered_ranges(u_c: np.ndarray, r: np.ndarray, c: float, n: int, chunk: int = 4096):
    """Vectorised ``covered_range`` over many records: returns lo, hi (-1 when empty)."""
    u_c = u_c.astype(np.float32)
    r = r.astype(np.float32)
    pix = np.arange(n, dtype=np.float32) - np.float32(c)
    lo = np.full(u_c.shape[0], -1, np.int64)
    hi = np.full(u_c.shape[0], -1, np.int64)
    for s in range(0, u_c.shape[0], chunk):
        cov = np.abs(u_c[s:s + chunk, None] - pix[None, :]) <= r[s:s + chunk, None]
        anyc = cov.any(axis=1)
        first = np.argmax(cov, axis=1)
        last = n - 1 - np.argmax(cov[:, ::-1], axis=1)
        lo[s:s + chunk] = np.where(anyc, first, -1)
        hi[s:s + chunk] = np.where(anyc, last, -1)
    return lo, hi


def reference_keys(records: np.ndarray, vis_bits: np.ndarray, view_of_rec: np.ndarray, cams: np.ndarray,
                   W: int, H: int, tw: int, th: int):
    """Per-bin sorted keys from the GPU's records: for every visible record, one
    key (FP32 depth bits << 32 | record) per tile its FP32 pixel window
    (|i - cx - uc| <= hx, |j - cy - vc| <= hy) touches; a stable sort of the
    keys by (bin, key).  Returns (bin_counts, keys_sorted)."""
    R = records.shape[0]
    bits = np.unpackbits(vis_bits.view(np.uint8), bitorder="little")[:R].astype(bool)
    rec = np.flatnonzero(bits)
    v = view_of_rec[rec]
    uc, vc, hx, hy, z = (records[rec, k] for k in (0, 1, 2, 3, 11))
    tiles_x, tiles_y = (W + tw - 1) // tw, (H + th - 1) // th
    tpv = tiles_x * tiles_y
    x_lo = np.empty(rec.size, np.int64)
    x_hi = np.empty(rec.size, np.int64)
    y_lo = np.empty(rec.size, np.int64)
    y_hi = np.empty(rec.size, np.int64)
    for vv in np.unique(v):
        s = v == vv
        x_lo[s], x_hi[s] = covered_ranges(uc[s], hx[s], cams[vv, 14], W)
        y_lo[s], y_hi[s] = covered_ranges(vc[s], hy[s], cams[vv, 15], H)
    assert np.all(x_lo >= 0) and np.all(y_lo >= 0), "a record marked visible covers no pixel"
    zbits = z.astype(np.float32).view(np.uint32).astype(np.uint64)
    key = (zbits << np.uint64(32)) | rec.astype(np.uint64)
    bins, keys = [], []
    bx0, bx1, by0, by1 = x_lo // tw, x_hi // tw, y_lo // th, y_hi // th
    nx, ny = bx1 - bx0 + 1, by1 - by0 + 1
    ntile = nx * ny
    rep = np.repeat(np.arange(rec.size), ntile)
    k = np.arange(ntile.sum()) - np.repeat(np.cumsum(ntile) - ntile, ntile)
    bx = bx0[rep] + k % nx[rep]
    by = by0[rep] + k // nx[rep]
    bins = v[rep].astype(np.int64) * tpv + by * tiles_x + bx
    keys = key[rep]
    order = np.lexsort((keys, bins))
    n_bins = int(view_of_rec.max(initial=0) + 1) * tpv if R else 0
    counts = np.bincount(bins, minlength=n_bins)
    return counts, keys[order]


def gpu_outputs(out, v=None):
    rgb, depth, T, nc = (t.detach().cpu().numpy() for t in out)
    if v is None:
        return dict(rgb=rgb, depth=depth, T=T, n_contrib=nc)
    return dict(rgb=rgb[v], depth=depth[v], T=T[v], n_contrib=nc[v])


GRAD_ELEM_REL = 1e-3  # per element: |g - g_ref| <= 1e-3 max|g_ref| + 1e-7 (per parameter group)
GRAD_ELEM_ABS = 1e-7


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def check_grad(a, b, name: str, rel_l2_max: float, elem_rel: float = GRAD_ELEM_REL,
               elem_abs: float = GRAD_ELEM_ABS) -> dict:
    """Gradient parity of one parameter group: the relative L2 error over the
    group is at most ``rel_l2_max``, and every element obeys
    |a - b| <= elem_rel * max|b| + elem_abs.  ``a`` is the CUDA result, ``b``
    the reference, both [N, ...] with N the Gaussian index (or any array).  The
    returned statistics (and the assertion message) name the worst element: its
    index (row = Gaussian), both values and the bound."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert a.shape == b.shape, (name, a.shape, b.shape)
    diff = np.abs(a - b)
    scale = float(np.abs(b).max(initial=0.0))
    bound = elem_rel * scale + elem_abs
    worst = int(np.argmax(diff)) if diff.size else 0
    idx = tuple(int(i) for i in np.unravel_index(worst, a.shape)) if diff.size else ()
    st = dict(group=name, rel_l2=rel_l2(a, b), worst_abs=float(diff.max(initial=0.0)), worst_index=idx,
              worst_value=float(a[idx]) if diff.size else 0.0, worst_ref=float(b[idx]) if diff.size else 0.0,
              elem_bound=bound, max_ref=scale, worst_over_bound=float(diff.max(initial=0.0)) / bound)
    print(f"grad {name}: rel L2 {st['rel_l2']:.2e}, worst |d| {st['worst_abs']:.2e} at {idx} "
          f"({st['worst_over_bound']:.3f} of the element bound)")
    assert st["rel_l2"] <= rel_l2_max, st
    assert st["worst_abs"] <= bound, st
    return st
