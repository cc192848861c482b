"""FP64 CPU oracle for the Gaussian-splatting RGB-D renderer and avatar LBS.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path (``paper_2604_12626_gb300``) never imports it,
and the two share no code: this package is plain C (``gs_oracle.c``, compiled
with gcc) plus NumPy marshalling.

Definitions followed (the paper cites tile-based 3DGS rasterisation for the
scene renderer, Sec. 2.2 and Sec. 3.2, and LBS deformation of canonical avatar
Gaussians by per-frame joint matrices, Sec. 3.1 and Sec. 3.3):

* ``project``  -- activation, view transform, EWA projection with the 0.3 px
  dilation, conic, 3-sigma radius, square footprint, SH degree-3 colour;
* ``render``   -- per-pixel front-to-back blending over covered Gaussians sorted
  by (FP32 depth key, index), alpha clamp 0.99, skip alpha < 1/255, stop before
  T < 1e-4; pixel-major brute force (``mode="pixel"``) or the equivalent
  Gaussian-major walk (``mode="gaussian"``); also returns the ambiguous-pixel
  mask (bit 1: value, bit 2: count) where FP32 rounding can flip a decision;
* ``render_backward`` -- the exact FP64 adjoint of ``render`` with its discrete
  decisions held fixed;
* ``lbs`` / ``lbs_backward`` -- linear blend skinning of means and covariances.

Parity of the whole pipeline against the paper's own renderer is unpinned: the
paper ships no code, data or printed values for it.  The pieces are pinned by
closed forms and invariants in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import contextlib
import ctypes
import hashlib
import os
import subprocess
import tempfile
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "gs_oracle.c"
_BUILD = _HERE / "_build"
_LIB = None

AMB_VALUE = 1
AMB_COUNT = 2
AMB_FOOTPRINT, AMB_ORDER, AMB_ALPHA, AMB_STOP = 4, 8, 16, 32  # which decision was near its threshold
AMB_CLAMP = 64  # alpha near the 0.99 clamp: the gradient (not the value) may differ


def _so_path() -> Path:
    h = hashlib.sha1(_SRC.read_bytes()).hexdigest()[:12]
    return _BUILD / f"liboracle_{h}.so"


def _compile(src: Path, out: Path) -> None:
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           str(src), "-o", str(out), "-lm"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C99 + OpenMP, FP contraction off)."""
    so = _so_path()
    if so.exists() and not force:
        return so
    _BUILD.mkdir(exist_ok=True)
    tmp = so.with_suffix(f".{os.getpid()}.tmp")
    _compile(_SRC, tmp)
    os.replace(tmp, so)
    return so


@contextlib.contextmanager
def variant(source: str):
    """Use a modified copy of the oracle source inside the block.  For the
    mutation tests, which plant a mistake and check that a pin catches it."""
    global _LIB
    with tempfile.TemporaryDirectory() as d:
        src, so = Path(d) / "mutant.c", Path(d) / "mutant.so"
        src.write_text(source)
        _compile(src, so)
        old = _LIB
        _LIB = _bind(ctypes.CDLL(str(so)))
        try:
            yield
        finally:
            _LIB = old


def source() -> str:
    return _SRC.read_text()


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = _bind(ctypes.CDLL(str(build())))
    return _LIB


def _bind(L):
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.or_project.restype = i64
    L.or_project.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, i32, i32, f64] + [P] * 12
    L.or_avatar_capsules.restype = None
    L.or_avatar_capsules.argtypes = [i32, i32, P, P, P, P, P]
    L.or_capsule_query.restype = None
    L.or_capsule_query.argtypes = [i64, P, P, P, P, P, f64, P, P, P, P]
    L.or_render.restype = i64
    L.or_render.argtypes = [i64, P, P, P, P, P, P, P, P, P, P, i32, i32, f64, P, i32, i32, i32] + [P] * 7
    L.or_lbs_matrices.restype = None
    L.or_lbs_matrices.argtypes = [i64, P, P, P, P, i32, P]
    L.or_render_backward.restype = i32
    L.or_render_backward.argtypes = [i64, P, P, P, P, P, P, P, P, i32, i32, f64, P, P, P] + [P] * 6
    L.or_lbs.restype = None
    L.or_lbs.argtypes = [i64, P, P, P, P, P, P, P, i32, P, P]
    L.or_lbs_backward.restype = None
    L.or_lbs_backward.argtypes = [i64, P, P, P, P, P, P, P, i32, P, P, P, P, P, P]
    L.or_sh_basis.restype = None
    L.or_sh_basis.argtypes = [i64, P, P]
    L.or_quat_to_rot.restype = None
    L.or_quat_to_rot.argtypes = [P, P]
    L.or_raster_mesh.restype = None
    L.or_raster_mesh.argtypes = [i64, P, P, i64, P, P, i32, i32, f64, P, P, P, P]
    L.or_composite_nearest.restype = None
    L.or_composite_nearest.argtypes = [i64, i64, P, P, P, P, P, P]
    L.or_forward_kinematics.restype = None
    L.or_forward_kinematics.argtypes = [i32, i32, P, P, P, P, P]
    L.or_interpolate_frames.restype = None
    L.or_interpolate_frames.argtypes = [i32, i32, i32, P, P, P]
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _u8(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _gauss(g: dict):
    n = int(np.asarray(g["means"]).shape[0])
    cov = _f64(g.get("cov3d"), (n, 6)) if g.get("cov3d") is not None else None
    use = _u8(g.get("use_cov")) if cov is not None else None
    if cov is not None and use is None:
        use = np.ones(n, np.uint8)
    return dict(
        n=n,
        means=_f64(g["means"], (n, 3)),
        log_scales=_f64(g["log_scales"], (n, 3)),
        quats=_f64(g["quats"], (n, 4)),
        ologits=_f64(g["opacity_logits"], (n,)),
        sh=_f64(g["sh"], (n, 16, 3)),
        cov3d=cov,
        use_cov=use,
        inexact=_u8(g.get("inexact")),
        dirmat=_f64(g.get("sh_dirmat"), (n, 9)) if g.get("sh_dirmat") is not None else None,
    )


def camera_array(R, C, fx, fy, cx, cy) -> np.ndarray:
    """Pack a camera as 16 float32 values: R (world->camera, row-major), C, fx, fy, cx, cy."""
    a = np.zeros(16, np.float32)
    a[:9] = np.asarray(R, np.float32).reshape(9)
    a[9:12] = np.asarray(C, np.float32).reshape(3)
    a[12:16] = [fx, fy, cx, cy]
    return a


def project(g: dict, cam, W: int, H: int, near: float = 0.2) -> dict:
    """Per-Gaussian projection into one view (FP64; FP32 depth key)."""
    L = _lib()
    G = _gauss(g)
    n = G["n"]
    cam64 = _f64(np.asarray(cam, np.float32))
    out = dict(
        visible=np.zeros(n, np.int32), u=np.zeros(n), v=np.zeros(n), z=np.zeros(n),
        zkey=np.zeros(n, np.float32), cov2=np.zeros((n, 3)), conic=np.zeros((n, 3)),
        opacity=np.zeros(n), rgb=np.zeros((n, 3)), radius=np.zeros(n, np.int32), r3=np.zeros(n),
        err=np.zeros((n, 6)),
    )
    L.or_project(n, _p(G["means"]), _p(G["log_scales"]), _p(G["quats"]), _p(G["ologits"]), _p(G["sh"]),
                 _p(G["cov3d"]), _p(G["use_cov"]), _p(G["inexact"]), _p(G["dirmat"]), _p(cam64), W, H, near,
                 _p(out["visible"]), _p(out["u"]), _p(out["v"]), _p(out["z"]), _p(out["zkey"]),
                 _p(out["cov2"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]),
                 _p(out["radius"]), _p(out["r3"]), _p(out["err"]))
    out["visible"] = out["visible"].astype(bool)
    # FP32 error bounds the ambiguity mask uses: of u, v (pixels), of 3 sqrt(lambda)
    # and of the conic entries A, B, C
    out["err_uv"], out["err_r3"], out["err_conic"] = out["err"][:, :2], out["err"][:, 2], out["err"][:, 3:6]
    return out


def render(g: dict, cam, W: int, H: int, near: float = 0.2, bg=(0.0, 0.0, 0.0), mode: str = "gaussian",
           normalize_depth: bool = False, nthreads: int = 0) -> dict:
    """Render one view.  Returns rgb [3,H,W], depth [H,W], T [H,W], n_contrib [H,W]
    (Gaussians blended into each pixel), n_covered [H,W] (covered Gaussians
    examined up to and including the last blended one), amb [H,W] (uint8 bit
    mask), last [H,W] (sorted position + 1 of the last blended Gaussian) and
    evals (covered Gaussians examined, the stopping one included)."""
    L = _lib()
    G = _gauss(g)
    cam64 = _f64(np.asarray(cam, np.float32))
    bg64 = _f64(bg)
    rgb = np.zeros((3, H, W))
    depth = np.zeros((H, W))
    T = np.zeros((H, W))
    ncon = np.zeros((H, W), np.int32)
    amb = np.zeros((H, W), np.uint8)
    last = np.zeros((H, W), np.int32)
    ncov = np.zeros((H, W), np.int32)
    ev = L.or_render(G["n"], _p(G["means"]), _p(G["log_scales"]), _p(G["quats"]), _p(G["ologits"]), _p(G["sh"]),
                     _p(G["cov3d"]), _p(G["use_cov"]), _p(G["inexact"]), _p(G["dirmat"]), _p(cam64), W, H, near,
                     _p(bg64),
                     0 if mode == "pixel" else 1, 1 if normalize_depth else 0, nthreads,
                     _p(rgb), _p(depth), _p(T), _p(ncon), _p(amb), _p(last), _p(ncov))
    return dict(rgb=rgb, depth=depth, T=T, n_contrib=ncon, n_covered=ncov, amb=amb, last=last, evals=int(ev))


def render_backward(g: dict, cam, W: int, H: int, d_rgb, d_depth, near: float = 0.2, bg=(0.0, 0.0, 0.0),
                    grads: dict | None = None) -> dict:
    """FP64 adjoint of ``render`` (raw depth).  Accumulates into ``grads`` if given."""
    L = _lib()
    G = _gauss(g)
    n = G["n"]
    if grads is None:
        grads = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                     opacity_logits=np.zeros(n), sh=np.zeros((n, 16, 3)),
                     cov3d=np.zeros((n, 6)) if G["cov3d"] is not None else None)
    cam64 = _f64(np.asarray(cam, np.float32))
    L.or_render_backward(n, _p(G["means"]), _p(G["log_scales"]), _p(G["quats"]), _p(G["ologits"]), _p(G["sh"]),
                         _p(G["cov3d"]), _p(G["use_cov"]), _p(cam64), W, H, near, _p(_f64(bg)),
                         _p(_f64(d_rgb, (3, H, W))), _p(_f64(d_depth, (H, W))),
                         _p(grads["means"]), _p(grads["log_scales"]), _p(grads["quats"]),
                         _p(grads["opacity_logits"]), _p(grads["sh"]), _p(grads.get("cov3d")))
    return grads


def lbs(means_c, log_scales_c, quats_c, joint_ids, weights, avatar_of, G):
    """Posed means [m,3] and covariances [m,6] (xx, xy, xz, yy, yz, zz)."""
    L = _lib()
    means_c = _f64(means_c)
    m = means_c.shape[0]
    G = _f64(G)
    nj = G.shape[1]
    ids = np.ascontiguousarray(np.asarray(joint_ids, np.int32).reshape(m, 4))
    av = np.ascontiguousarray(np.asarray(avatar_of, np.int32).reshape(m))
    om, oc = np.zeros((m, 3)), np.zeros((m, 6))
    L.or_lbs(m, _p(means_c), _p(_f64(log_scales_c)), _p(_f64(quats_c)), _p(ids), _p(_f64(weights)), _p(av),
             _p(G), nj, _p(om), _p(oc))
    return om, oc


def lbs_matrices(joint_ids, weights, avatar_of, G):
    """The blended skinning matrices A [m,3,4] of the avatar Gaussians."""
    L = _lib()
    G = _f64(G)
    nj = G.shape[1]
    ids = np.ascontiguousarray(np.asarray(joint_ids, np.int32).reshape(-1, 4))
    m = ids.shape[0]
    av = np.ascontiguousarray(np.asarray(avatar_of, np.int32).reshape(m))
    out = np.zeros((m, 3, 4))
    L.or_lbs_matrices(m, _p(ids), _p(_f64(weights)), _p(av), _p(G), nj, _p(out))
    return out


def lbs_backward(means_c, log_scales_c, quats_c, joint_ids, weights, avatar_of, G, g_means, g_cov):
    """Gradients w.r.t. canonical means, log-scales, quaternions and joint matrices."""
    L = _lib()
    means_c = _f64(means_c)
    m = means_c.shape[0]
    G = _f64(G)
    nj = G.shape[1]
    ids = np.ascontiguousarray(np.asarray(joint_ids, np.int32).reshape(m, 4))
    av = np.ascontiguousarray(np.asarray(avatar_of, np.int32).reshape(m))
    out = dict(means=np.zeros((m, 3)), log_scales=np.zeros((m, 3)), quats=np.zeros((m, 4)), G=np.zeros(G.shape))
    L.or_lbs_backward(m, _p(means_c), _p(_f64(log_scales_c)), _p(_f64(quats_c)), _p(ids), _p(_f64(weights)),
                      _p(av), _p(G), nj, _p(_f64(g_means)), _p(_f64(g_cov)), _p(out["means"]),
                      _p(out["log_scales"]), _p(out["quats"]), _p(out["G"]))
    return out


def raster_mesh(verts, colors, tris, cam, W: int, H: int, near: float = 0.2, bg=(0.0, 0.0, 0.0)) -> dict:
    """z-buffered triangle mesh layer: rgb [3,H,W], depth [H,W] (0 where
    uncovered), amb [H,W] (1 where FP32 rounding could change the pixel)."""
    L = _lib()
    v = _f64(verts)
    tr = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(-1, 3))
    rgb, depth, amb = np.zeros((3, H, W)), np.zeros((H, W)), np.zeros((H, W), np.uint8)
    L.or_raster_mesh(v.shape[0], _p(v), _p(_f64(colors)), tr.shape[0], _p(tr), _p(_f64(np.asarray(cam, np.float32))),
                     W, H, near, _p(_f64(bg)), _p(rgb), _p(depth), _p(amb))
    return dict(rgb=rgb, depth=depth, amb=amb)


def composite_nearest(rgb_a, depth_a, rgb_b, depth_b):
    """Nearest-fragment composite of two layers: rgb [V,3,H,W], depth [V,H,W]."""
    L = _lib()
    da, db = _f64(depth_a), _f64(depth_b)
    V = da.shape[0] if da.ndim == 3 else 1
    hw = da.size // V
    rgb = np.zeros((V, 3) + da.shape[-2:])
    dep = np.zeros((V,) + da.shape[-2:])
    L.or_composite_nearest(V, hw, _p(_f64(rgb_a)), _p(da), _p(_f64(rgb_b)), _p(db), _p(rgb), _p(dep))
    return rgb, dep


def forward_kinematics(local_rot, root, rest, parents):
    """Skinning matrices [A,J,3,4] from local rotations [A,J,3,3], root [A,3,4],
    rest joints [J,3] and parents [J]."""
    L = _lib()
    lr = _f64(local_rot)
    A, J = lr.shape[0], lr.shape[1]
    out = np.zeros((A, J, 3, 4))
    par = np.ascontiguousarray(np.asarray(parents, np.int32).reshape(J))
    L.or_forward_kinematics(A, J, _p(lr), _p(_f64(root)), _p(_f64(rest)), _p(par), _p(out))
    return out


def avatar_capsules(M, rest, parents, radius):
    """Proxy capsules [A,J,8] (a xyz, rho, b xyz, 0) from skinning matrices
    M [A,J,3,4]: joint j's capsule spans the posed parent and j (the root: a
    sphere), posed position = M_j [J_j; 1]."""
    L = _lib()
    Mm = _f64(M)
    A, J = Mm.shape[0], Mm.shape[1]
    out = np.zeros((A, J, 8))
    par = np.ascontiguousarray(np.asarray(parents, np.int32).reshape(J))
    L.or_avatar_capsules(A, J, _p(Mm), _p(_f64(rest)), _p(par), _p(_f64(radius)), _p(out))
    return out


def capsule_query(caps, env_cap_off, query_env, p0, p1=None, agent_radius=0.0):
    """Per query: signed distance from p0 to the nearest capsule surface of its
    env, that capsule's index within the env (-1: none), and for the step
    p0 -> p1 the first-contact fraction tclip and the blocked flag."""
    L = _lib()
    c = _f64(caps).reshape(-1, 8)
    off = np.ascontiguousarray(np.asarray(env_cap_off, np.int64))
    qe = np.ascontiguousarray(np.asarray(query_env, np.int32))
    Q = qe.shape[0]
    P0 = _f64(p0).reshape(Q, 3)
    P1 = None if p1 is None else _f64(p1).reshape(Q, 3)
    dist = np.zeros(Q)
    near = np.zeros(Q, np.int32)
    tclip = np.zeros(Q)
    blk = np.zeros(Q, np.uint8)
    L.or_capsule_query(Q, _p(c), _p(off), _p(qe), _p(P0), _p(P1) if P1 is not None else None, float(agent_radius),
                       _p(dist), _p(near), _p(tclip), _p(blk))
    return dict(dist=dist, nearest=near, tclip=tclip, blocked=blk.astype(bool))


def interpolate_frames(frames, t):
    """Joint matrices [A,J,3,4] at fractional frame positions t [A] from frames [A,F,J,3,4]."""
    L = _lib()
    fr = _f64(frames)
    A, F, J = fr.shape[0], fr.shape[1], fr.shape[2]
    out = np.zeros((A, J, 3, 4))
    L.or_interpolate_frames(A, F, J, _p(fr), _p(_f64(np.asarray(t, np.float64).reshape(A))), _p(out))
    return out


def sh_basis(dirs) -> np.ndarray:
    """Real SH basis (degree 3, 16 functions) at unit directions [n,3]."""
    L = _lib()
    d = _f64(dirs).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16))
    L.or_sh_basis(d.shape[0], _p(d), _p(out))
    return out


def quat_to_rot(q) -> np.ndarray:
    L = _lib()
    q = _f64(q).reshape(4)
    R = np.zeros(9)
    L.or_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def render_views(g: dict, cams, W: int, H: int, **kw) -> list:
    """Render several views of one scene (one call per view)."""
    return [render(g, c, W, H, **kw) for c in cams]
