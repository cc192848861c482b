"""Seeded synthetic inputs for the renderer: indoor-room scenes, cameras and
Gaussian avatars with a 24-joint kinematic tree.

This module draws inputs only; it holds none of the rendering or skinning
arithmetic.  It serves the CUDA path, the CPU oracle, the tests and the
benchmark alike.  All arrays are float32 (indices int32/uint16), laid out as
the renderer expects: means [N,3], log_scales [N,3], quats [N,4] (w, x, y, z,
not normalised), opacity_logits [N], sh [N,16,3] (coefficient-major, channel
fastest).

The paper evaluates on real 3DGS scans (InteriorGS, reconstructions; Sec. 4.1)
at 256x256 with 300K-7M Gaussians and 0-10 avatars (Sec. 4.5, Table 6).  Those
assets are not available here; the generators below stand in for them with the
same sizes and an indoor structure: most Gaussians are flat splats on the
room's floor, walls and ceiling, the rest are furniture-like blobs.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOM = (10.0, 8.0, 3.0)  # metres, z up
CAMERA_HEIGHT = 1.2

# SMPL-like 24-joint tree: parent of each joint, rest positions (x lateral,
# y forward, z up) relative to the pelvis, in metres (about 1.7 m tall).
PARENTS = np.array([-1, 0, 0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 9, 9, 12, 13, 14, 16, 17, 18, 19, 20, 21], np.int32)
REST_JOINTS = np.array([
    [0.00, 0.00, 0.00], [0.09, 0.00, -0.08], [-0.09, 0.00, -0.08], [0.00, 0.00, 0.11],
    [0.10, 0.00, -0.46], [-0.10, 0.00, -0.46], [0.00, 0.00, 0.25], [0.10, 0.00, -0.86],
    [-0.10, 0.00, -0.86], [0.00, 0.00, 0.31], [0.10, 0.12, -0.91], [-0.10, 0.12, -0.91],
    [0.00, 0.00, 0.52], [0.07, 0.00, 0.43], [-0.07, 0.00, 0.43], [0.00, 0.00, 0.70],
    [0.18, 0.00, 0.45], [-0.18, 0.00, 0.45], [0.44, 0.00, 0.45], [-0.44, 0.00, 0.45],
    [0.69, 0.00, 0.45], [-0.69, 0.00, 0.45], [0.77, 0.00, 0.45], [-0.77, 0.00, 0.45],
], np.float64)
N_JOINTS = 24


def _normal(rng, shape, mean=0.0, std=1.0):
    x = rng.standard_normal(size=shape, dtype=np.float32)
    if std != 1.0:
        x *= np.float32(std)
    if mean != 0.0:
        x += np.float32(mean)
    return x


def _appearance(rng, n: int, g: dict) -> dict:
    """Opacity logits ~ N(0,1); SH DC ~ N(0,0.3), bands 1-3 ~ N(0,0.05)."""
    g["opacity_logits"] = _normal(rng, (n,))
    sh = _normal(rng, (n, 16, 3), std=0.05)
    sh[:, 0, :] = _normal(rng, (n, 3), std=0.3)
    g["sh"] = sh
    return g


def _random_quats(rng, n: int) -> np.ndarray:
    q = _normal(rng, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    w1, x1, y1, z1 = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    w2, x2, y2, z2 = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=-1)


def box_scene(n: int = 5000, seed: int = 0) -> dict:
    """Gaussians uniform in [-1,1]x[-1,1]x[2,6] (camera space of an identity
    camera), log-scales N(-3.5, 0.5), random unit quaternions."""
    rng = np.random.default_rng(seed)
    g = {}
    m = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    m[:, 0] = m[:, 0] * 2 - 1
    m[:, 1] = m[:, 1] * 2 - 1
    m[:, 2] = m[:, 2] * 4 + 2
    g["means"] = m
    g["log_scales"] = _normal(rng, (n, 3), -3.5, 0.5)
    g["quats"] = _random_quats(rng, n)
    return _appearance(rng, n, g)


# plane: (axis of the normal, coordinate, area)
_PLANES = [(2, 0.0, 80.0), (2, ROOM[2], 80.0), (0, 0.0, 24.0), (0, ROOM[0], 24.0), (1, 0.0, 30.0), (1, ROOM[1], 30.0)]
_S2 = math.sqrt(0.5)
# quaternion taking local z onto the plane normal axis
_PLANE_Q = {2: np.array([1.0, 0.0, 0.0, 0.0]), 0: np.array([_S2, 0.0, _S2, 0.0]), 1: np.array([_S2, -_S2, 0.0, 0.0])}


def room_scene(n: int = 1_000_000, seed: int = 0, planar_frac: float = 0.7, n_clusters: int = 20) -> dict:
    """Indoor room [0,10]x[0,8]x[0,3] m.  ``planar_frac`` of the Gaussians lie
    on the six room planes (plane chosen by area, offset U(-2,2) cm along the
    normal, log-scales N(-4, 0.6) with the normal axis shrunk by 3, normal-
    aligned frame with a random in-plane spin); the rest form ``n_clusters``
    isotropic blobs of sigma 0.3 m (centres in the room shrunk by 0.5 m,
    clipped to the room, random rotations, log-scales N(-4, 0.6))."""
    rng = np.random.default_rng(seed)
    n_pl = int(round(n * planar_frac))
    n_cl = n - n_pl
    means = np.empty((n, 3), np.float32)
    ls = _normal(rng, (n, 3), -4.0, 0.6)
    quats = np.empty((n, 4), np.float32)
    areas = np.array([p[2] for p in _PLANES])
    which = rng.choice(len(_PLANES), size=n_pl, p=areas / areas.sum())
    uvw = rng.uniform(0.0, 1.0, size=(n_pl, 3))
    pts = uvw * np.array(ROOM)
    off = rng.uniform(-0.02, 0.02, size=n_pl)
    spin = rng.uniform(0.0, 2.0 * math.pi, size=n_pl)
    qspin = np.stack([np.cos(spin / 2), np.zeros(n_pl), np.zeros(n_pl), np.sin(spin / 2)], axis=1)
    for k, (ax, coord, _a) in enumerate(_PLANES):
        sel = which == k
        pts[sel, ax] = coord + off[sel]
        quats[:n_pl][sel] = _quat_mul(np.broadcast_to(_PLANE_Q[ax], (int(sel.sum()), 4)), qspin[sel]).astype(np.float32)
    means[:n_pl] = pts.astype(np.float32)
    ls[:n_pl, 2] -= np.float32(3.0)
    lo = np.array([0.5, 0.5, 0.5])
    hi = np.array(ROOM) - 0.5
    centres = rng.uniform(lo, hi, size=(n_clusters, 3))
    cid = rng.integers(0, n_clusters, size=n_cl)
    blob = centres[cid] + rng.standard_normal(size=(n_cl, 3)) * 0.3
    blob = np.clip(blob, 0.0, np.array(ROOM))
    means[n_pl:] = blob.astype(np.float32)
    quats[n_pl:] = _random_quats(rng, n_cl)
    g = {"means": means, "log_scales": ls, "quats": quats}
    return _appearance(rng, n, g)


def look_camera(position, yaw: float, W: int, H: int, hfov_deg: float = 90.0, pitch: float = 0.0) -> np.ndarray:
    """Camera as 16 float32: R (world->camera rows: right, down, forward; OpenCV
    convention in a z-up world), centre C, fx, fy, cx, cy.  Pixel (i, j) has its
    centre at (i, j), so the principal point is ((W-1)/2, (H-1)/2)."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    fwd = np.array([cy_ * cp, sy_ * cp, sp])
    right = np.array([sy_, -cy_, 0.0])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    f = 0.5 * W / math.tan(math.radians(hfov_deg) / 2)
    cam = np.zeros(16, np.float32)
    cam[:9] = R.reshape(9)
    cam[9:12] = position
    cam[12:16] = [f, f, (W - 1) / 2.0, (H - 1) / 2.0]
    return cam


def identity_camera(W: int, H: int, hfov_deg: float = 90.0) -> np.ndarray:
    cam = np.zeros(16, np.float32)
    cam[:9] = np.eye(3, dtype=np.float32).reshape(9)
    f = 0.5 * W / math.tan(math.radians(hfov_deg) / 2)
    cam[12:16] = [f, f, (W - 1) / 2.0, (H - 1) / 2.0]
    return cam


def room_camera(seed: int, W: int, H: int, hfov_deg: float = 90.0) -> np.ndarray:
    """Random pose inside the room at 1.2 m height with a random yaw."""
    rng = np.random.default_rng(10_000 + seed)
    pos = [rng.uniform(0.5, ROOM[0] - 0.5), rng.uniform(0.5, ROOM[1] - 0.5), CAMERA_HEIGHT]
    return look_camera(pos, rng.uniform(0.0, 2.0 * math.pi), W, H, hfov_deg)


def concat(scenes: list) -> tuple:
    """Concatenate per-env Gaussian dicts; returns (arrays, env_offsets [E+1])."""
    keys = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    out = {k: np.concatenate([s[k] for s in scenes], axis=0) for k in keys}
    offs = np.zeros(len(scenes) + 1, np.int64)
    offs[1:] = np.cumsum([s["means"].shape[0] for s in scenes])
    return out, offs


def batched_rooms(n_envs: int = 64, n_min: int = 300_000, n_max: int = 1_500_000, W: int = 256, H: int = 256,
                  seed0: int = 0, scale: float = 1.0):
    """One room per env (env e seeded by seed0 + e) with N_e ~ U{n_min..n_max}
    (times ``scale``), one camera per env.  Returns (arrays, env_offsets, cams)."""
    sizes = batch_sizes(n_envs, n_min, n_max, seed0, scale)
    with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 4)) as ex:  # the generators release the GIL
        scenes = list(ex.map(lambda e: room_scene(sizes[e], seed=seed0 + e), range(n_envs)))
    cams = [room_camera(seed0 + e, W, H) for e in range(n_envs)]
    g, offs = concat(scenes)
    return g, offs, np.stack(cams)


def batch_sizes(n_envs: int = 64, n_min: int = 300_000, n_max: int = 1_500_000, seed0: int = 0, scale: float = 1.0):
    """The per-env Gaussian counts ``batched_rooms`` draws, without drawing the scenes."""
    return [max(int(np.random.default_rng(seed0 + e).integers(n_min, n_max + 1) * scale), 1) for e in range(n_envs)]


# ---------------------------------------------------------------------------
# Triangle meshes (the mesh layer of a mixed scene)
# ---------------------------------------------------------------------------

def room_mesh(seed: int = 0, n_boxes: int = 12, grid: int = 8) -> dict:
    """A triangle mesh of the room: its six faces, each a grid x grid quad
    mesh, and n_boxes axis-aligned boxes (furniture) on the floor; random
    per-vertex colours.  vertices [V,3], colors [V,3] float32, triangles
    [T,3] int32."""
    rng = np.random.default_rng(60_000 + seed)
    verts, tris = [], []

    def add_quad_grid(origin, u, v, n):
        base = sum(len(x) for x in verts)
        a = np.linspace(0.0, 1.0, n + 1)
        pts = origin[None, None, :] + a[:, None, None] * u[None, None, :] + a[None, :, None] * v[None, None, :]
        verts.append(pts.reshape(-1, 3))
        for i in range(n):
            for j in range(n):
                k = base + i * (n + 1) + j
                tris.append([k, k + n + 1, k + n + 2])
                tris.append([k, k + n + 2, k + 1])

    X, Y, Z = ROOM
    e = np.eye(3)
    faces = [(np.zeros(3), X * e[0], Y * e[1]), (np.array([0, 0, Z]), X * e[0], Y * e[1]),
             (np.zeros(3), X * e[0], Z * e[2]), (np.array([0, Y, 0]), X * e[0], Z * e[2]),
             (np.zeros(3), Y * e[1], Z * e[2]), (np.array([X, 0, 0]), Y * e[1], Z * e[2])]
    for o, u, v in faces:
        add_quad_grid(np.asarray(o, np.float64), u, v, grid)
    for _ in range(n_boxes):
        size = rng.uniform([0.3, 0.3, 0.3], [1.5, 1.5, 1.2])
        lo = np.array([rng.uniform(0.2, X - 0.2 - size[0]), rng.uniform(0.2, Y - 0.2 - size[1]), 0.0])
        hi = lo + size
        for axis in range(3):
            for side in (lo, hi):
                o = lo.copy()
                o[axis] = side[axis]
                a1, a2 = [k for k in range(3) if k != axis]
                add_quad_grid(o, (hi - lo)[a1] * e[a1], (hi - lo)[a2] * e[a2], 1)
    V = np.concatenate(verts).astype(np.float32)
    return {"vertices": V, "colors": rng.uniform(0.0, 1.0, (V.shape[0], 3)).astype(np.float32),
            "triangles": np.asarray(tris, np.int32)}


# ---------------------------------------------------------------------------
# Avatars
# ---------------------------------------------------------------------------

def avatar_canonical(n: int = 50_000, seed: int = 0) -> dict:
    """Canonical (rest-pose) avatar Gaussians within 8 cm of the bone segments
    of the 24-joint tree, log-scales N(-4.5, 0.3); 4 distinct skin joints drawn
    uniformly from 0..23 per Gaussian with Dirichlet(1,1,1,1) weights."""
    rng = np.random.default_rng(50_000 + seed)
    bones = [(j, int(PARENTS[j])) for j in range(1, N_JOINTS)]
    lens = np.array([np.linalg.norm(REST_JOINTS[a] - REST_JOINTS[b]) + 0.05 for a, b in bones])
    bi = rng.choice(len(bones), size=n, p=lens / lens.sum())
    t = rng.uniform(0.0, 1.0, size=n)
    a = REST_JOINTS[[bones[k][0] for k in bi]]
    b = REST_JOINTS[[bones[k][1] for k in bi]]
    pts = a + (b - a) * t[:, None]
    d = rng.standard_normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = 0.08 * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    pts += d * rad[:, None]
    g = {"means": pts.astype(np.float32), "log_scales": _normal(rng, (n, 3), -4.5, 0.3), "quats": _random_quats(rng, n)}
    _appearance(rng, n, g)
    ids = np.argsort(rng.uniform(0.0, 1.0, size=(n, N_JOINTS)), axis=1)[:, :4]
    g["joint_ids"] = ids.astype(np.uint16)
    g["weights"] = rng.dirichlet(np.ones(4), size=n).astype(np.float32)
    return g


def rodrigues(aa: np.ndarray) -> np.ndarray:
    """Rotation matrices [..., 3, 3] from axis-angle vectors [..., 3]."""
    th = np.linalg.norm(aa, axis=-1, keepdims=True)
    k = np.where(th > 1e-12, aa / np.maximum(th, 1e-12), 0.0)
    K = np.zeros(aa.shape[:-1] + (3, 3))
    K[..., 0, 1], K[..., 0, 2] = -k[..., 2], k[..., 1]
    K[..., 1, 0], K[..., 1, 2] = k[..., 2], -k[..., 0]
    K[..., 2, 0], K[..., 2, 1] = -k[..., 1], k[..., 0]
    s = np.sin(th)[..., None]
    c = np.cos(th)[..., None]
    return np.eye(3) + s * K + (1 - c) * (K @ K)


def forward_kinematics(theta: np.ndarray, root_t, yaw: float = 0.0) -> np.ndarray:
    """Skinning matrices [24, 3, 4] of the synthetic tree: G_0 = [Rz(yaw) Rod(theta_0) | t],
    G_j = G_parent [Rod(theta_j) | J_j - J_parent], M_j = G_j [I | -J_j]."""
    Rz = rodrigues(np.array([0.0, 0.0, yaw]))
    Rl = rodrigues(np.asarray(theta, np.float64).reshape(N_JOINTS, 3))
    GR = np.zeros((N_JOINTS, 3, 3))
    Gt = np.zeros((N_JOINTS, 3))
    GR[0] = Rz @ Rl[0]
    Gt[0] = np.asarray(root_t, np.float64)
    for j in range(1, N_JOINTS):
        p = PARENTS[j]
        GR[j] = GR[p] @ Rl[j]
        Gt[j] = GR[p] @ (REST_JOINTS[j] - REST_JOINTS[p]) + Gt[p]
    M = np.zeros((N_JOINTS, 3, 4))
    M[:, :, :3] = GR
    M[:, :, 3] = Gt - np.einsum("jab,jb->ja", GR, REST_JOINTS)
    return M


def random_pose(seed: int, root_t=None, sigma: float = 0.3) -> np.ndarray:
    """Joint matrices [24,3,4] for axis-angle theta ~ N(0, sigma) per component,
    root translation uniform in the room at z = 0.9 and a random yaw."""
    rng = np.random.default_rng(70_000 + seed)
    theta = rng.normal(0.0, sigma, size=(N_JOINTS, 3))
    if root_t is None:
        root_t = [rng.uniform(0.5, ROOM[0] - 0.5), rng.uniform(0.5, ROOM[1] - 0.5), 0.9]
    return forward_kinematics(theta, root_t, rng.uniform(0.0, 2.0 * math.pi)).astype(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even); returns the uint16 bit patterns."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    return ((u + r) >> 16).astype(np.uint16)


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


def training_scene(seed: int = 0, n_room: int = 500_000, n_avatars: int = 2, n_per: int = 50_000,
                   n_views: int = 16, W: int = 512, H: int = 512) -> dict:
    """The forward + backward training workload: one room of ``n_room``
    Gaussians, ``n_avatars`` avatars of ``n_per`` Gaussians (24-joint tree,
    posed per frame with theta ~ N(0, 0.3)), ``n_views`` cameras at random poses
    (hfov 90 degrees, so f = W / 2 at 512 px: 256), avatar a standing 2 m in
    front of camera a so that the joint transforms are seen; and the
    perturbation of the target scene: means + N(0, 1 cm), SH + N(0, 0.02), for
    the room's and the avatars' canonical Gaussians alike.  Returns a dict:
    room (Gaussian dict), avatars (canonical dict with joint_ids, weights,
    avatar_of), G [A,24,3,4], cams [V,16], d_room_means, d_room_sh,
    d_av_means, d_av_sh (float32)."""
    rng = np.random.default_rng(80_000 + seed)
    room = room_scene(n_room, seed=seed)
    avs = [avatar_canonical(n_per, 100 * seed + a) for a in range(n_avatars)]
    av = {k: np.concatenate([a[k] for a in avs]) for k in avs[0]}
    av["avatar_of"] = np.repeat(np.arange(n_avatars), n_per).astype(np.int32)
    cams = np.stack([room_camera(1000 * seed + v, W, H) for v in range(n_views)])
    G = np.stack([random_pose(1000 * seed + a) for a in range(n_avatars)]).astype(np.float32)
    for a in range(n_avatars):
        fwd, C = cams[a % n_views][6:9].astype(np.float64), cams[a % n_views][9:12].astype(np.float64)
        root = C + 2.0 * fwd + np.array([0.0, 0.0, -0.3])
        G[a, :, :, 3] += (root - G[a, 0, :, 3]).astype(np.float32)
    return dict(room=room, avatars=av, G=G, cams=cams,
                d_room_means=_normal(rng, (n_room, 3), 0.0, 0.01), d_room_sh=_normal(rng, (n_room, 16, 3), 0.0, 0.02),
                d_av_means=_normal(rng, (n_avatars * n_per, 3), 0.0, 0.01),
                d_av_sh=_normal(rng, (n_avatars * n_per, 16, 3), 0.0, 0.02))
