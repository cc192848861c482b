"""Thin ctypes binding of libgs (include/gs.h) plus the torch.autograd.Function.

Argument marshalling only: every step of the renderer runs in libgs's CUDA
kernels.  PyTorch provides device memory (workspaces, outputs) and streams.
There is no CPU fallback: importing this module raises if libgs.so has not been
built, and every call raises on a non-zero status.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np
import torch

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libgs.so"
if not _LIB_PATH.exists():
    raise ImportError(f"libgs.so is not built ({_LIB_PATH}); run `python -m paper_2604_12626_gb300.build`")
_lib = ctypes.CDLL(str(_LIB_PATH))

GS_OK = 0
STATUS_NAMES = {0: "GS_OK", -1: "GS_ERR_INVALID_ARG", -2: "GS_ERR_ALIGNMENT", -3: "GS_ERR_WORKSPACE_TOO_SMALL",
                -4: "GS_ERR_CAPACITY", -5: "GS_ERR_CUDA", -6: "GS_ERR_TIMEOUT", -7: "GS_ERR_UNSUPPORTED"}
SH_F32, SH_F16, SH_BF16 = 0, 1, 2
FLAG_PERSISTENT, FLAG_NORMALIZE_DEPTH, FLAG_GRAD_OVERWRITE, FLAG_COUNT_EVALS, FLAG_AVATAR_CANONICAL_SH = 1, 2, 4, 8, 16
FLAG_GRAD_PRECLEARED = 32
N_STAGES = 11
STAGES = ("setup", "preprocess", "scan", "scatter", "sort", "merge", "blend", "blend_backward",
          "preprocess_backward", "deform", "deform_backward")
MAX_ENVS = MAX_VIEWS = 512

_P = ctypes.c_void_p


class GsCamera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("C", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class GsGaussians(ctypes.Structure):
    _fields_ = [("means", _P), ("log_scales", _P), ("quats", _P), ("opacity_logits", _P), ("sh", _P),
                ("sh_dtype", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cov3d", _P), ("n", ctypes.c_int64)]


class GsBatch(ctypes.Structure):
    _fields_ = [("n_envs", ctypes.c_int32), ("n_views", ctypes.c_int32), ("env_offsets", _P),
                ("env_cov3d_begin", _P), ("view_env", _P)]


class GsRenderConfig(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("batch_depth", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("bg", ctypes.c_float * 3), ("near_plane", ctypes.c_float), ("pair_capacity", ctypes.c_int64),
                ("pix_x", ctypes.c_int32), ("pix_y", ctypes.c_int32)]


class GsStats(ctypes.Structure):
    _fields_ = [("n_records", ctypes.c_int64), ("n_visible", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("max_bin", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_evaluations", ctypes.c_int64), ("n_covered", ctypes.c_int64)]


class GsWsSections(ctypes.Structure):
    _fields_ = [("records", _P), ("vis", _P), ("keys", _P), ("bin_start", _P), ("quarters", _P),
                ("n_records", ctypes.c_int64),
                ("pair_capacity", ctypes.c_int64), ("n_bins", ctypes.c_int32), ("tiles_x", ctypes.c_int32),
                ("tiles_y", ctypes.c_int32), ("tiles_per_view", ctypes.c_int32)]


class GsAvatars(ctypes.Structure):
    _fields_ = [("means", _P), ("log_scales", _P), ("quats", _P), ("joint_ids", _P), ("weights", _P),
                ("avatar_of", _P), ("dest", _P), ("m", ctypes.c_int64), ("n_avatars", ctypes.c_int32),
                ("n_joints", ctypes.c_int32)]


class GsMesh(ctypes.Structure):
    _fields_ = [("vertices", _P), ("colors", _P), ("triangles", _P), ("n_vertices", ctypes.c_int64),
                ("n_triangles", ctypes.c_int64)]


_R = ctypes.POINTER
_lib.gs_render_workspace_size.argtypes = [_R(GsRenderConfig), _R(GsBatch), _R(ctypes.c_size_t)]
_lib.gs_render.argtypes = [_R(GsGaussians), _R(GsBatch), _P, _R(GsRenderConfig), _P, ctypes.c_size_t, _P, _P, _P, _P,
                           _P]
_lib.gs_render_backward.argtypes = [_R(GsGaussians), _R(GsBatch), _P, _R(GsRenderConfig), _P, ctypes.c_size_t, _P, _P,
                                    _P, _P, _P, _P, _P, _P, _P]
_lib.gs_deform_avatars.argtypes = [_R(GsAvatars), _P, _P, _P, _P]
_lib.gs_render_avatars.argtypes = [_R(GsGaussians), _R(GsBatch), _R(GsAvatars), _P, _P, _R(GsRenderConfig), _P,
                                   ctypes.c_size_t, _P, _P, _P, _P, _P]
_lib.gs_render_avatars_backward.argtypes = [_R(GsGaussians), _R(GsBatch), _R(GsAvatars), _P, _P, _R(GsRenderConfig),
                                            _P, ctypes.c_size_t] + [_P] * 13
_lib.gs_render_avatars_backward.restype = ctypes.c_int32
_lib.gs_zero_gradients.argtypes = [ctypes.c_int64, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]
_lib.gs_zero_gradients.restype = ctypes.c_int32
_lib.gs_mesh_workspace_size.argtypes = [_R(GsBatch), _R(ctypes.c_size_t)]
_lib.gs_render_mesh.argtypes = [_R(GsMesh), _R(GsBatch), _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_float, _P,
                                ctypes.c_size_t, _P, _P, _P]
_lib.gs_composite_nearest.argtypes = [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]
_lib.gs_forward_kinematics.argtypes = [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]
_lib.gs_interpolate_joints.argtypes = [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P]
_lib.gs_deform_avatars_backward.argtypes = [_R(GsAvatars), _P, _P, _P, _P, _P, _P, _P, _P]
_lib.gs_get_status.argtypes = [_P, ctypes.c_size_t, _P, _R(ctypes.c_int32)]
_lib.gs_render_stats.argtypes = [_P, ctypes.c_size_t, _P, _R(GsStats)]
_lib.gs_autotune.argtypes = [_R(GsGaussians), _R(GsBatch), _P, _R(GsRenderConfig), _P, ctypes.c_size_t, _P, _P, _P,
                             _P, _P, ctypes.c_int32, ctypes.c_int32, _R(ctypes.c_float), _P]
_lib.gs_workspace_sections.argtypes = [_R(GsRenderConfig), _R(GsBatch), _P, _R(GsWsSections)]
_lib.gs_render_static.argtypes = [_R(GsGaussians), _R(GsBatch), _P, _R(GsRenderConfig), _P, _P, _P, _P, _P]
_lib.gs_render_static_status.argtypes = [_P, _R(ctypes.c_int32)]
_lib.gs_profile_enable.argtypes = [ctypes.c_int32]
_lib.gs_profile_read.argtypes = [_P, _P]
for _f in ("gs_render_static", "gs_render_static_status", "gs_profile_enable", "gs_profile_read", "gs_workspace_sections", "gs_render_workspace_size", "gs_render", "gs_render_backward", "gs_deform_avatars",
           "gs_deform_avatars_backward", "gs_get_status", "gs_render_stats", "gs_autotune"):
    getattr(_lib, _f).restype = ctypes.c_int32
_lib.gs_exp2_rate.argtypes = [ctypes.c_int32, ctypes.c_int32, _P, _P]
_lib.gs_avatar_capsules.argtypes = [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]
_lib.gs_avatar_capsules.restype = ctypes.c_int32
_lib.gs_capsule_query.argtypes = [_P, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_float, ctypes.c_int64, _P, _P, _P, _P,
                                  _P]
_lib.gs_capsule_query.restype = ctypes.c_int32
_lib.gs_exp2_rate.restype = ctypes.c_int32
_lib.gs_last_cuda_error.restype = ctypes.c_int32
_lib.gs_version.restype = ctypes.c_int32

EXPORTS = ("gs_render_static", "gs_render_static_status", "gs_profile_enable", "gs_profile_read", "gs_workspace_sections", "gs_render_workspace_size", "gs_render", "gs_render_backward", "gs_deform_avatars",
           "gs_deform_avatars_backward", "gs_get_status", "gs_render_stats", "gs_autotune", "gs_last_cuda_error",
           "gs_version", "gs_composite_nearest", "gs_forward_kinematics", "gs_interpolate_joints",
           "gs_render_avatars", "gs_render_avatars_backward", "gs_mesh_workspace_size", "gs_render_mesh",
           "gs_exp2_rate", "gs_avatar_capsules", "gs_capsule_query", "gs_zero_gradients")


class GsError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != GS_OK:
        extra = f" (cudaError {_lib.gs_last_cuda_error()})" if st == -5 else ""
        raise GsError(f"{what} failed: {STATUS_NAMES.get(st, st)}{extra}")


def lib_path() -> str:
    return str(_LIB_PATH)


def version() -> int:
    return _lib.gs_version()


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _sh_dtype(t: torch.Tensor) -> int:
    return {torch.float32: SH_F32, torch.float16: SH_F16, torch.bfloat16: SH_BF16}[t.dtype]


def _need(t, dtype, shape_tail, name):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}")


class Batch:
    """Batch structure: env_offsets [E+1], view_env [V], optional env_cov3d_begin [E] (host arrays)."""

    def __init__(self, env_offsets, view_env=None, env_cov3d_begin=None):
        self.env_offsets = np.ascontiguousarray(np.asarray(env_offsets, np.int64))
        E = len(self.env_offsets) - 1
        self.view_env = np.ascontiguousarray(np.asarray(view_env if view_env is not None else np.arange(E), np.int32))
        self.env_cov3d_begin = (None if env_cov3d_begin is None else
                                np.ascontiguousarray(np.asarray(env_cov3d_begin, np.int64)))
        self.c = GsBatch(E, len(self.view_env), self.env_offsets.ctypes.data_as(_P),
                         None if self.env_cov3d_begin is None else self.env_cov3d_begin.ctypes.data_as(_P),
                         self.view_env.ctypes.data_as(_P))

    @property
    def n_envs(self):
        return len(self.env_offsets) - 1

    @property
    def n_views(self):
        return len(self.view_env)

    @property
    def n_gaussians(self):
        return int(self.env_offsets[-1])


def profile_enable(on: bool = True):
    _check(_lib.gs_profile_enable(1 if on else 0), "gs_profile_enable")


def profile_read() -> dict:
    """Per-stage (summed ms, launches) since the last read; synchronises."""
    ms = (ctypes.c_float * N_STAGES)()
    n = (ctypes.c_int32 * N_STAGES)()
    _check(_lib.gs_profile_read(ctypes.cast(ms, _P), ctypes.cast(n, _P)), "gs_profile_read")
    return {STAGES[i]: (ms[i], n[i]) for i in range(N_STAGES) if n[i]}


def make_config(width, height, tile=(16, 16), batch_depth=256, bg=(0.0, 0.0, 0.0), near=0.2, pair_capacity=0,
                persistent=False, normalize_depth=False, grad_overwrite=False, pix=(1, 1)) -> GsRenderConfig:
    c = GsRenderConfig()
    c.width, c.height = width, height
    c.tile_w, c.tile_h = tile
    c.pix_x, c.pix_y = pix
    c.batch_depth = batch_depth
    c.flags = ((FLAG_PERSISTENT if persistent else 0) | (FLAG_NORMALIZE_DEPTH if normalize_depth else 0)
               | (FLAG_GRAD_OVERWRITE if grad_overwrite else 0))
    c.bg[:] = list(bg)
    c.near_plane = near
    c.pair_capacity = pair_capacity
    return c


def workspace_size(cfg: GsRenderConfig, batch: Batch) -> int:
    n = ctypes.c_size_t(0)
    _check(_lib.gs_render_workspace_size(ctypes.byref(cfg), ctypes.byref(batch.c), ctypes.byref(n)),
           "gs_render_workspace_size")
    return n.value


def cameras_tensor(cams: np.ndarray, device="cuda") -> torch.Tensor:
    """[V,16] float32 (R, C, fx, fy, cx, cy) -> device tensor laid out as gs_camera[V]."""
    a = np.ascontiguousarray(np.asarray(cams, np.float32).reshape(-1, 16))
    return torch.from_numpy(a).to(device)


class Gaussians:
    """Device tensors of the concatenated Gaussians (see gs_gaussians)."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh, cov3d=None):
        n = means.shape[0]
        _need(means, torch.float32, (3,), "means")
        _need(log_scales, torch.float32, (3,), "log_scales")
        _need(quats, torch.float32, (4,), "quats")
        _need(opacity_logits, torch.float32, (), "opacity_logits")
        if sh.dtype not in (torch.float32, torch.float16, torch.bfloat16):
            raise ValueError("sh must be float32, float16 or bfloat16")
        _need(sh, sh.dtype, (16, 3), "sh")
        if cov3d is not None:
            _need(cov3d, torch.float32, (6,), "cov3d")
        for t in (log_scales, quats, opacity_logits, sh):
            if t.shape[0] != n:
                raise ValueError("all Gaussian arrays need the same length")
        self.means, self.log_scales, self.quats, self.opacity_logits, self.sh, self.cov3d = (
            means, log_scales, quats, opacity_logits, sh, cov3d)
        self.c = GsGaussians(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                             _sh_dtype(sh), 0, _ptr(cov3d), n)

    @classmethod
    def from_numpy(cls, g: dict, device="cuda", sh_dtype=torch.float32):
        t = {k: torch.from_numpy(np.ascontiguousarray(g[k])).to(device) for k in
             ("means", "log_scales", "quats", "opacity_logits", "sh")}
        sh = t["sh"].to(sh_dtype)
        cov = None
        if g.get("cov3d") is not None:
            cov = torch.from_numpy(np.ascontiguousarray(g["cov3d"], np.float32)).to(device)
        return cls(t["means"], t["log_scales"], t["quats"], t["opacity_logits"], sh, cov)


class Renderer:
    """A configured renderer with its own workspace (one gs_render / gs_render_backward pair)."""

    def __init__(self, batch: Batch, width: int, height: int, device="cuda", tile_candidates=None, **cfg_kw):
        """``tile_candidates``: (tile_w, tile_h, batch_depth, pix_x, pix_y)
        rows the workspace must also fit (for autotune over them)."""
        self.batch = batch
        self.cfg = make_config(width, height, **cfg_kw)
        self.device = torch.device(device)
        self.ws_bytes = workspace_size(self.cfg, batch)
        for c in tile_candidates or ():
            k = dict(cfg_kw, tile=(c[0], c[1]), batch_depth=c[2], pix=(c[3], c[4]))
            self.ws_bytes = max(self.ws_bytes, workspace_size(make_config(width, height, **k), batch))
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.workspace[:4096].zero_()  # status word and counters

    @property
    def width(self):
        return self.cfg.width

    @property
    def height(self):
        return self.cfg.height

    def alloc_outputs(self):
        V, H, W = self.batch.n_views, self.cfg.height, self.cfg.width
        dev = self.device
        return (torch.empty((V, 3, H, W), device=dev), torch.empty((V, H, W), device=dev),
                torch.empty((V, H, W), device=dev), torch.empty((V, H, W), dtype=torch.int32, device=dev))

    def forward(self, g: Gaussians, cams: torch.Tensor, out=None, stream=None):
        """Returns (rgb [V,3,H,W], depth [V,H,W], T [V,H,W], n_contrib [V,H,W])."""
        if out is None:
            out = self.alloc_outputs()
        rgb, depth, T, nc = out
        _check(_lib.gs_render(ctypes.byref(g.c), ctypes.byref(self.batch.c), _ptr(cams), ctypes.byref(self.cfg),
                              _ptr(self.workspace), self.ws_bytes, _ptr(rgb), _ptr(depth), _ptr(T), _ptr(nc),
                              _stream(stream)), "gs_render")
        return out

    def backward(self, g: Gaussians, cams: torch.Tensor, d_rgb, d_depth, grads=None, stream=None,
                 precleared: bool = False):
        """Adds dL/d(params) into ``grads`` (allocated zero if None), or
        overwrites them in overwrite mode; returns it.  ``precleared``: the
        arrays were set to zero beforehand (zero_gradients, e.g. on a stream
        beside the forward), so the backward writes the seen rows only."""
        n = g.means.shape[0]
        dev = self.device
        if grads is None:
            grads = dict(means=torch.zeros((n, 3), device=dev), log_scales=torch.zeros((n, 3), device=dev),
                         quats=torch.zeros((n, 4), device=dev), opacity_logits=torch.zeros((n,), device=dev),
                         sh=torch.zeros((n, 16, 3), device=dev),
                         cov3d=torch.zeros((n, 6), device=dev) if g.cov3d is not None else None)
        d_rgb = d_rgb.contiguous()
        d_depth = d_depth.contiguous()
        cfg = GsRenderConfig.from_buffer_copy(self.cfg)
        if precleared:
            cfg.flags |= FLAG_GRAD_PRECLEARED
        _check(_lib.gs_render_backward(ctypes.byref(g.c), ctypes.byref(self.batch.c), _ptr(cams),
                                       ctypes.byref(cfg), _ptr(self.workspace), self.ws_bytes, _ptr(d_rgb),
                                       _ptr(d_depth), _ptr(grads["means"]), _ptr(grads["log_scales"]),
                                       _ptr(grads["quats"]), _ptr(grads["opacity_logits"]), _ptr(grads["sh"]),
                                       _ptr(grads.get("cov3d")), _stream(stream)), "gs_render_backward")
        return grads

    def forward_avatars(self, g: Gaussians, av: "Avatars", joint_G: torch.Tensor, cams: torch.Tensor, out=None,
                        stream=None):
        """gs_render_avatars: like forward, with the avatar rows of every env
        (from the batch's env_cov3d_begin on) posed by LBS inside the
        preprocess from ``av`` (canonical rows in env order, no dest)."""
        if out is None:
            out = self.alloc_outputs()
        rgb, depth, T, nc = out
        _check(_lib.gs_render_avatars(ctypes.byref(g.c), ctypes.byref(self.batch.c), ctypes.byref(av.c),
                                      _ptr(joint_G), _ptr(cams), ctypes.byref(self.cfg), _ptr(self.workspace),
                                      self.ws_bytes, _ptr(rgb), _ptr(depth), _ptr(T), _ptr(nc), _stream(stream)),
               "gs_render_avatars")
        return out

    def backward_avatars(self, g: Gaussians, av: "Avatars", joint_G: torch.Tensor, cams: torch.Tensor, d_rgb, d_depth,
                         grads=None, avatar_grads=None, stream=None):
        """gs_render_avatars_backward after forward_avatars: ``grads`` as for
        backward (all rows; an avatar row's mean and cov3d entries hold the
        posed gradients), ``avatar_grads`` (canonical means, log_scales, quats
        and the joint matrices G) added to.  Both allocated zero if None."""
        n, m = g.means.shape[0], av.m
        dev = self.device
        if grads is None:
            grads = dict(means=torch.zeros((n, 3), device=dev), log_scales=torch.zeros((n, 3), device=dev),
                         quats=torch.zeros((n, 4), device=dev), opacity_logits=torch.zeros((n,), device=dev),
                         sh=torch.zeros((n, 16, 3), device=dev), cov3d=torch.zeros((n, 6), device=dev))
        if avatar_grads is None:
            avatar_grads = dict(means=torch.zeros((m, 3), device=dev), log_scales=torch.zeros((m, 3), device=dev),
                                quats=torch.zeros((m, 4), device=dev), G=torch.zeros_like(joint_G))
        d_rgb = d_rgb.contiguous()
        d_depth = d_depth.contiguous()
        _check(_lib.gs_render_avatars_backward(
            ctypes.byref(g.c), ctypes.byref(self.batch.c), ctypes.byref(av.c), _ptr(joint_G), _ptr(cams),
            ctypes.byref(self.cfg), _ptr(self.workspace), self.ws_bytes, _ptr(d_rgb), _ptr(d_depth),
            _ptr(grads["means"]), _ptr(grads["log_scales"]), _ptr(grads["quats"]), _ptr(grads["opacity_logits"]),
            _ptr(grads["sh"]), _ptr(grads["cov3d"]), _ptr(avatar_grads["means"]), _ptr(avatar_grads["log_scales"]),
            _ptr(avatar_grads["quats"]), _ptr(avatar_grads["G"]), _stream(stream)), "gs_render_avatars_backward")
        return grads, avatar_grads

    def stats(self, stream=None) -> dict:
        s = GsStats()
        _check(_lib.gs_render_stats(_ptr(self.workspace), self.ws_bytes, _stream(stream), ctypes.byref(s)),
               "gs_render_stats")
        return dict(n_records=s.n_records, n_visible=s.n_visible, n_pairs=s.n_pairs, max_bin=s.max_bin,
                    status=s.status, n_evaluations=s.n_evaluations, n_covered=s.n_covered)

    def count_evaluations(self, g: Gaussians, cams: torch.Tensor, out=None, stream=None) -> int:
        """Runs one forward with GS_FLAG_COUNT_EVALS and returns the blend
        evaluations (per pixel, the covered Gaussians examined up to and
        including the one that stops it, summed over all views); the stats
        then also hold n_covered (per pixel, the covered Gaussians up to and
        including the last blended one, summed)."""
        prev = self.cfg.flags
        self.cfg.flags = prev | FLAG_COUNT_EVALS
        try:
            self.forward(g, cams, out=out, stream=stream)
            return self.stats(stream)["n_evaluations"]
        finally:
            self.cfg.flags = prev

    def status(self, stream=None) -> int:
        v = ctypes.c_int32(0)
        _check(_lib.gs_get_status(_ptr(self.workspace), self.ws_bytes, _stream(stream), ctypes.byref(v)),
               "gs_get_status")
        return v.value

    def sections(self) -> dict:
        """Views into the workspace left by the last forward: records [R,12] float32,
        vis [ceil(R/32)] int32 bits, keys [cap] int64 (depth bits << 32 | record; bit 31 set
        by the blend on pairs some pixel of the tile blended),
        bin_start [n_bins+1] int32, quarters [cap] int32 at 2 x 1 pixels per thread
        (else None: per flagged pair, byte w = the quarters of warp w that blended
        it), plus the tile grid."""
        s = GsWsSections()
        _check(_lib.gs_workspace_sections(ctypes.byref(self.cfg), ctypes.byref(self.batch.c), _ptr(self.workspace),
                                          ctypes.byref(s)), "gs_workspace_sections")
        base = self.workspace.data_ptr()

        def view(addr, nbytes, dtype):
            off = addr - base
            return self.workspace[off:off + nbytes].view(dtype)

        R = s.n_records
        return dict(records=view(s.records, R * 48, torch.float32).view(R, 12),
                    vis=view(s.vis, ((R + 31) // 32) * 4, torch.int32),
                    keys=view(s.keys, s.pair_capacity * 8, torch.int64),
                    bin_start=view(s.bin_start, (s.n_bins + 1) * 4, torch.int32),
                    quarters=view(s.quarters, s.pair_capacity * 4, torch.int32) if s.quarters else None,
                    n_bins=s.n_bins, tiles_x=s.tiles_x, tiles_y=s.tiles_y, tiles_per_view=s.tiles_per_view,
                    pair_capacity=s.pair_capacity)

    def kernels_per_forward(self) -> int:
        """Kernel launches of one forward: setup, preprocess, scan, scatter,
        the two sorts, one merge pass per doubling of 4096 up to the largest
        possible bin (the pair capacity or the most records of one view), blend."""
        cap = self.sections()["pair_capacity"]
        offs = self.batch.env_offsets
        max_view = max(int(offs[e + 1] - offs[e]) for e in self.batch.view_env)
        chunks = -(-min(cap, max_view) // 4096)
        return 7 + max(0, (chunks - 1).bit_length())

    def autotune(self, g: Gaussians, cams: torch.Tensor, candidates, reps=3, out=None, stream=None):
        """Time each (tile_w, tile_h, batch_depth, pix_x, pix_y) candidate; keep the fastest in self.cfg."""
        if out is None:
            out = self.alloc_outputs()
        cand = np.ascontiguousarray(np.asarray(candidates, np.int32).reshape(-1, 5))
        best = ctypes.c_float(0)
        cfg = GsRenderConfig.from_buffer_copy(self.cfg)
        rgb, depth, T, nc = out
        _check(_lib.gs_autotune(ctypes.byref(g.c), ctypes.byref(self.batch.c), _ptr(cams), ctypes.byref(cfg),
                                _ptr(self.workspace), self.ws_bytes, _ptr(rgb), _ptr(depth), _ptr(T), _ptr(nc),
                                cand.ctypes.data_as(_P), len(cand), reps, ctypes.byref(best), _stream(stream)),
               "gs_autotune")
        self.cfg = cfg
        return (cfg.tile_w, cfg.tile_h, cfg.batch_depth, cfg.pix_x, cfg.pix_y), best.value


class Avatars:
    """Canonical avatar Gaussians and skinning data on the device (see gs_avatars)."""

    def __init__(self, means, log_scales, quats, joint_ids, weights, avatar_of, n_avatars, n_joints=24, dest=None):
        m = means.shape[0]
        _need(means, torch.float32, (3,), "means")
        _need(log_scales, torch.float32, (3,), "log_scales")
        _need(quats, torch.float32, (4,), "quats")
        _need(weights, torch.float32, (4,), "weights")
        if joint_ids.dtype != torch.int16 or tuple(joint_ids.shape) != (m, 4):
            raise ValueError("joint_ids must be [M,4] int16 (uint16 bit pattern)")
        if avatar_of.dtype != torch.int32 or tuple(avatar_of.shape) != (m,):
            raise ValueError("avatar_of must be [M] int32")
        if dest is not None and (dest.dtype != torch.int64 or tuple(dest.shape) != (m,)):
            raise ValueError("dest must be [M] int64")
        self.t = (means, log_scales, quats, joint_ids, weights, avatar_of, dest)
        self.m, self.n_avatars, self.n_joints = m, n_avatars, n_joints
        self.c = GsAvatars(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(joint_ids), _ptr(weights),
                           _ptr(avatar_of), _ptr(dest), m, n_avatars, n_joints)


STATIC_SCRATCH_BYTES = 64 << 20


def render_static(g: Gaussians, batch: Batch, cams: torch.Tensor, cfg: GsRenderConfig, out, stream=None):
    """gs_render_static: a forward render that allocates nothing (scratch in a
    64 MiB static device array inside libgs).  ``out`` = (rgb, depth, T,
    n_contrib) preallocated by the caller.  Calls must not overlap on the GPU."""
    rgb, depth, T, nc = out
    _check(_lib.gs_render_static(ctypes.byref(g.c), ctypes.byref(batch.c), _ptr(cams), ctypes.byref(cfg), _ptr(rgb),
                                 _ptr(depth), _ptr(T), _ptr(nc), _stream(stream)), "gs_render_static")
    return out


def render_static_status(stream=None) -> int:
    """gs_render_static_status: synchronises; the device status word the last
    gs_render_static call left (0 or GS_ERR_CAPACITY = -4), then cleared."""
    v = ctypes.c_int32(0)
    _check(_lib.gs_render_static_status(_stream(stream), ctypes.byref(v)), "gs_render_static_status")
    return v.value


def zero_gradients(grads: dict, n_ctas: int = 0, stream=None):
    """gs_zero_gradients: sets the arrays of ``grads`` (means, log_scales, quats,
    opacity_logits, sh, optional cov3d) to zero with TMA bulk stores from
    ``n_ctas`` CTAs (0: one per two SMs), asynchronously on ``stream``."""
    n = grads["means"].shape[0]
    _check(_lib.gs_zero_gradients(n, _ptr(grads["means"]), _ptr(grads["log_scales"]), _ptr(grads["quats"]),
                                  _ptr(grads["opacity_logits"]), _ptr(grads["sh"]), _ptr(grads.get("cov3d")),
                                  int(n_ctas), _stream(stream)), "gs_zero_gradients")
    return grads


def deform(av: Avatars, G: torch.Tensor, out_means: torch.Tensor, out_cov3d: torch.Tensor, stream=None):
    _check(_lib.gs_deform_avatars(ctypes.byref(av.c), _ptr(G), _ptr(out_means), _ptr(out_cov3d), _stream(stream)),
           "gs_deform_avatars")


def deform_backward(av: Avatars, G, d_means, d_cov3d, grads, stream=None):
    _check(_lib.gs_deform_avatars_backward(ctypes.byref(av.c), _ptr(G), _ptr(d_means), _ptr(d_cov3d),
                                           _ptr(grads["means"]), _ptr(grads["log_scales"]), _ptr(grads["quats"]),
                                           _ptr(grads["G"]), _stream(stream)), "gs_deform_avatars_backward")
    return grads


class Mesh:
    """A triangle mesh with per-vertex colours on the device (see gs_mesh)."""

    def __init__(self, vertices, colors, triangles):
        _need(vertices, torch.float32, (3,), "vertices")
        _need(colors, torch.float32, (3,), "colors")
        if triangles.dtype != torch.int32 or triangles.dim() != 2 or triangles.shape[1] != 3:
            raise ValueError("triangles must be [T,3] int32")
        self.t = (vertices, colors, triangles)
        self.c = GsMesh(_ptr(vertices), _ptr(colors), _ptr(triangles), vertices.shape[0], triangles.shape[0])

    @staticmethod
    def from_numpy(m: dict, device="cuda"):
        T = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x)).to(device, dt)  # noqa: E731
        return Mesh(T(m["vertices"], torch.float32), T(m["colors"], torch.float32),
                    T(m["triangles"], torch.int32))


def render_mesh(mesh: Mesh, batch: Batch, cams: torch.Tensor, width: int, height: int, bg=(0.0, 0.0, 0.0),
                near: float = 0.2, out=None, workspace=None, stream=None):
    """The mesh layer (gs_render_mesh): (rgb [V,3,H,W], depth [V,H,W]); batch
    env_offsets index triangles."""
    nbytes = ctypes.c_size_t(0)
    _check(_lib.gs_mesh_workspace_size(ctypes.byref(batch.c), ctypes.byref(nbytes)), "gs_mesh_workspace_size")
    dev = cams.device
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(max(int(nbytes.value), 16), dtype=torch.uint8, device=dev)
    V = batch.n_views
    if out is None:
        out = (torch.empty((V, 3, height, width), device=dev), torch.empty((V, height, width), device=dev))
    bg3 = (ctypes.c_float * 3)(*bg)
    _check(_lib.gs_render_mesh(ctypes.byref(mesh.c), ctypes.byref(batch.c), _ptr(cams), width, height, bg3, near,
                               _ptr(workspace), workspace.numel(), _ptr(out[0]), _ptr(out[1]), _stream(stream)),
           "gs_render_mesh")
    return out


def exp2_rate(n_blocks: int, iters: int, out: torch.Tensor, stream=None) -> int:
    """gs_exp2_rate: launches the exp2 throughput kernel (out: float32 CUDA
    tensor of n_blocks * 256); returns the exp2 operations it performs."""
    if out.dtype != torch.float32 or not out.is_cuda or out.numel() < n_blocks * 256:
        raise GsError("exp2_rate: float32 CUDA tensor of n_blocks * 256 expected")
    _check(_lib.gs_exp2_rate(n_blocks, iters, _ptr(out), _stream(stream)), "gs_exp2_rate")
    return n_blocks * 256 * iters * 8


def composite_nearest(rgb_a, depth_a, rgb_b, depth_b, out=None, stream=None):
    """Per pixel the nearer of two RGB-D layers (gs_composite_nearest).
    rgb [V,3,H,W], depth [V,H,W] float32 CUDA tensors; returns (rgb, depth)."""
    V, _, H, W = rgb_a.shape
    for t, shp in ((rgb_a, (V, 3, H, W)), (rgb_b, (V, 3, H, W)), (depth_a, (V, H, W)), (depth_b, (V, H, W))):
        if tuple(t.shape) != shp or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise GsError("composite_nearest: contiguous float32 CUDA tensors [V,3,H,W] and [V,H,W] expected")
    if out is None:
        out = (torch.empty_like(rgb_a), torch.empty_like(depth_a))
    _check(_lib.gs_composite_nearest(_ptr(rgb_a), _ptr(depth_a), _ptr(rgb_b), _ptr(depth_b), V, H, W, _ptr(out[0]),
                                     _ptr(out[1]), _stream(stream)), "gs_composite_nearest")
    return out


def forward_kinematics(local_rot, root, rest, parents, out=None, stream=None):
    """Skinning matrices [A,J,3,4] (gs_forward_kinematics) from local rotations
    [A,J,3,3], root [A,3,4] and rest joints [J,3] (CUDA float32) and the parent
    of each joint (host sequence)."""
    A, J = local_rot.shape[0], local_rot.shape[1]
    par = np.ascontiguousarray(np.asarray(parents, np.int32).reshape(J))
    if out is None:
        out = torch.empty((A, J, 3, 4), dtype=torch.float32, device=local_rot.device)
    _check(_lib.gs_forward_kinematics(_ptr(local_rot), _ptr(root), _ptr(rest), par.ctypes.data_as(_P), A, J,
                                      _ptr(out), _stream(stream)), "gs_forward_kinematics")
    return out


def avatar_capsules(joint_M, rest, parents, radius, out=None, stream=None):
    """Proxy capsules [A,J,8] (a xyz, radius, b xyz, 0; gs_avatar_capsules) of
    avatars posed by skinning matrices joint_M [A,J,3,4]: joint j's capsule
    spans the posed parent and j.  rest [J,3], radius [J] CUDA float32; parents
    a host sequence."""
    A, J = joint_M.shape[0], joint_M.shape[1]
    _need(joint_M, torch.float32, (J, 3, 4), "joint_M")
    _need(rest, torch.float32, (3,), "rest")
    _need(radius, torch.float32, (), "radius")
    par = np.ascontiguousarray(np.asarray(parents, np.int32).reshape(J))
    if out is None:
        out = torch.empty((A, J, 8), dtype=torch.float32, device=joint_M.device)
    _check(_lib.gs_avatar_capsules(_ptr(joint_M), _ptr(rest), par.ctypes.data_as(_P), _ptr(radius), A, J, _ptr(out),
                                   _stream(stream)), "gs_avatar_capsules")
    return out


def capsule_query(caps, env_cap_off, query_env, p0, p1=None, agent_radius=0.0, out=None, stream=None):
    """The avatar queries (gs_capsule_query): per query, the signed distance
    from p0 to the nearest capsule surface of its env, that capsule's row
    within the env, and for the step p0 -> p1 the first-contact fraction and
    the blocked flag.  caps [C,8], env_cap_off [E+1] int64, query_env [Q] int32,
    p0 / p1 [Q,3]: CUDA tensors.  Returns (dist, nearest, tclip, blocked)."""
    Q = query_env.shape[0]
    _need(caps, torch.float32, (8,), "caps")
    _need(env_cap_off, torch.int64, (), "env_cap_off")
    _need(query_env, torch.int32, (), "query_env")
    _need(p0, torch.float32, (3,), "p0")
    if p1 is not None:
        _need(p1, torch.float32, (3,), "p1")
    if out is None:
        dev = p0.device
        out = (torch.empty(Q, dtype=torch.float32, device=dev), torch.empty(Q, dtype=torch.int32, device=dev),
               torch.empty(Q, dtype=torch.float32, device=dev), torch.empty(Q, dtype=torch.uint8, device=dev))
    dist, near, tclip, blk = out
    _check(_lib.gs_capsule_query(_ptr(caps), _ptr(env_cap_off), env_cap_off.shape[0] - 1, _ptr(query_env), _ptr(p0),
                                 _ptr(p1) if p1 is not None else None, float(agent_radius), Q, _ptr(dist),
                                 _ptr(near), _ptr(tclip), _ptr(blk), _stream(stream)), "gs_capsule_query")
    return out


def interpolate_joints(frames, t, out=None, stream=None):
    """Joint matrices [A,J,3,4] at fractional frame positions t [A] from
    per-frame matrices [A,F,J,3,4] (gs_interpolate_joints)."""
    A, F, J = frames.shape[0], frames.shape[1], frames.shape[2]
    if out is None:
        out = torch.empty((A, J, 3, 4), dtype=torch.float32, device=frames.device)
    _check(_lib.gs_interpolate_joints(_ptr(frames), _ptr(t), A, F, J, _ptr(out), _stream(stream)),
           "gs_interpolate_joints")
    return out


class RenderFunction(torch.autograd.Function):
    """(means, log_scales, quats, opacity_logits, sh) -> (rgb [V,3,H,W], depth [V,H,W]).

    The forward runs gs_render; the backward runs gs_render_backward with the
    per-pixel (T_final, last index) checkpoint kept in the renderer workspace.
    SH gradients are float32 whatever the SH storage type."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, renderer: Renderer, cams):
        g = Gaussians(means.detach(), log_scales.detach(), quats.detach(), opacity_logits.detach(), sh.detach())
        rgb, depth, T, nc = renderer.forward(g, cams)
        ctx.renderer, ctx.cams, ctx.g = renderer, cams, g
        ctx.sh_dtype = sh.dtype
        return rgb, depth

    @staticmethod
    def backward(ctx, d_rgb, d_depth):
        r = ctx.renderer
        V, H, W = r.batch.n_views, r.height, r.width
        if d_rgb is None:
            d_rgb = torch.zeros((V, 3, H, W), device=r.device)
        if d_depth is None:
            d_depth = torch.zeros((V, H, W), device=r.device)
        gr = r.backward(ctx.g, ctx.cams, d_rgb.float(), d_depth.float())
        return (gr["means"], gr["log_scales"], gr["quats"], gr["opacity_logits"], gr["sh"].to(ctx.sh_dtype), None,
                None)


def render(means, log_scales, quats, opacity_logits, sh, renderer: Renderer, cams):
    """Differentiable batched render; see RenderFunction."""
    return RenderFunction.apply(means, log_scales, quats, opacity_logits, sh, renderer, cams)


class AvatarScene:
    """One env of scene Gaussians plus avatars posed by LBS every frame,
    rendered jointly in one pass into the env's views (Sec. 3.2 last
    paragraph, Sec. 3.3), with every buffer allocated once so that a forward +
    backward training step captures into one CUDA graph.

    Rows: the scene's Gaussians, then the avatars' (their mean and covariance
    written by gs_deform_avatars each forward).  ``scene``: device tensors
    means, log_scales, quats, opacity_logits, sh of the scene; ``avatars``:
    canonical means, log_scales, quats, opacity_logits, sh plus joint_ids
    ([M,4] int16 holding the uint16 ids), weights, avatar_of (int32).  They
    are copied into this object's own concatenated tensors (``scene_params`` /
    ``avatar_params`` are views of them, to be updated in place by an
    optimizer).  Gradients: gs_render_backward in overwrite mode into
    ``grads`` (all rows), then gs_deform_avatars_backward into ``avatar_grads``
    (canonical means, log_scales, quats and the joint transforms G).  With
    ``fused`` the avatars are posed inside the render instead
    (gs_render_avatars / gs_render_avatars_backward): nothing posed is written
    to memory and the same gradients come out."""

    def __init__(self, scene: dict, avatars: dict, n_avatars: int, n_joints: int, width: int, height: int,
                 n_views: int, sh_dtype=torch.float32, device="cuda", fused: bool = False, **cfg_kw):
        dev = torch.device(device)
        ns, m = scene["means"].shape[0], avatars["means"].shape[0]
        n = ns + m
        self.ns, self.m, self.n_avatars, self.n_joints = ns, m, n_avatars, n_joints
        f32 = dict(device=dev, dtype=torch.float32)
        self.means = torch.empty((n, 3), **f32)
        self.means[:ns] = scene["means"]
        self.log_scales = torch.zeros((n, 3), **f32)
        self.log_scales[:ns] = scene["log_scales"]
        self.quats = torch.zeros((n, 4), **f32)
        self.quats[:ns] = scene["quats"]
        self.quats[ns:, 0] = 1.0
        self.opacity_logits = torch.cat([scene["opacity_logits"], avatars["opacity_logits"]]).to(**f32).contiguous()
        self.sh = torch.cat([scene["sh"], avatars["sh"]]).to(device=dev, dtype=sh_dtype).contiguous()
        self.cov3d = torch.zeros((n, 6), **f32)
        self.av_means = avatars["means"].to(**f32).clone().contiguous()
        self.av_log_scales = avatars["log_scales"].to(**f32).clone().contiguous()
        self.av_quats = avatars["quats"].to(**f32).clone().contiguous()
        self.av = Avatars(self.av_means, self.av_log_scales, self.av_quats, avatars["joint_ids"].contiguous(),
                          avatars["weights"].to(**f32).contiguous(), avatars["avatar_of"].contiguous(), n_avatars,
                          n_joints, dest=torch.arange(ns, n, dtype=torch.int64, device=dev))
        self.g = Gaussians(self.means, self.log_scales, self.quats, self.opacity_logits, self.sh, self.cov3d)
        self.fused = fused
        if fused:  # canonical rows in env order (one env), no posed covariance
            self.av_fused = Avatars(self.av_means, self.av_log_scales, self.av_quats, self.av.t[3], self.av.t[4],
                                    self.av.t[5], n_avatars, n_joints)
            self.g_fused = Gaussians(self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)
        batch = Batch(np.array([0, n]), view_env=np.zeros(n_views, np.int32), env_cov3d_begin=[ns])
        self.renderer = Renderer(batch, width, height, device=device, grad_overwrite=True, **cfg_kw)
        self.out = self.renderer.alloc_outputs()
        self.grads = dict(means=torch.empty((n, 3), **f32), log_scales=torch.empty((n, 3), **f32),
                          quats=torch.empty((n, 4), **f32), opacity_logits=torch.empty((n,), **f32),
                          sh=torch.empty((n, 16, 3), **f32), cov3d=torch.empty((n, 6), **f32))
        self.avatar_grads = dict(means=torch.empty((m, 3), **f32), log_scales=torch.empty((m, 3), **f32),
                                 quats=torch.empty((m, 4), **f32),
                                 G=torch.empty((n_avatars, n_joints, 3, 4), **f32))

    @property
    def scene_params(self) -> dict:
        ns = self.ns
        return dict(means=self.means[:ns], log_scales=self.log_scales[:ns], quats=self.quats[:ns],
                    opacity_logits=self.opacity_logits[:ns], sh=self.sh[:ns])

    @property
    def avatar_params(self) -> dict:
        return dict(means=self.av_means, log_scales=self.av_log_scales, quats=self.av_quats,
                    opacity_logits=self.opacity_logits[self.ns:], sh=self.sh[self.ns:])

    def forward(self, G: torch.Tensor, cams: torch.Tensor, stream=None):
        """Poses the avatars with joint transforms G [A,J,3,4] and renders every
        view: (rgb, depth, T, n_contrib) in this object's output buffers."""
        if self.fused:
            return self.renderer.forward_avatars(self.g_fused, self.av_fused, G, cams, out=self.out, stream=stream)
        deform(self.av, G, self.means, self.cov3d, stream=stream)
        return self.renderer.forward(self.g, cams, out=self.out, stream=stream)

    def backward(self, G: torch.Tensor, cams: torch.Tensor, d_rgb: torch.Tensor, d_depth: torch.Tensor, stream=None):
        """Adjoint of the last forward: (grads of every row, canonical avatar
        grads with dL/dG).  Scene rows of ``grads`` are the scene's gradients,
        avatar rows of its opacity_logits / sh the avatars' own."""
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            for t in self.avatar_grads.values():
                t.zero_()
        if self.fused:
            self.renderer.backward_avatars(self.g_fused, self.av_fused, G, cams, d_rgb, d_depth, grads=self.grads,
                                           avatar_grads=self.avatar_grads, stream=stream)
            return self.grads, self.avatar_grads
        self.renderer.backward(self.g, cams, d_rgb, d_depth, grads=self.grads, stream=stream)
        deform_backward(self.av, G, self.grads["means"], self.grads["cov3d"], self.avatar_grads, stream=stream)
        return self.grads, self.avatar_grads


class SceneWithAvatarsFunction(torch.autograd.Function):
    """Scene Gaussians plus LBS-deformed avatar Gaussians rendered in one pass.

    Inputs: scene (means, log_scales, quats, opacity_logits, sh) [Ns...], avatar
    canonical (means, log_scales, quats) [M...], avatar opacity_logits [M], avatar
    sh [M,16,3], joint matrices G [A,J,3,4].  One env: Gaussian order is scene then
    avatars.  Gradients flow to all of them, including G, through
    gs_deform_avatars_backward."""

    @staticmethod
    def forward(ctx, s_means, s_ls, s_q, s_op, s_sh, a_means, a_ls, a_q, a_op, a_sh, G, av_static, renderer, cams):
        ns, m = s_means.shape[0], a_means.shape[0]
        dev = s_means.device
        means = torch.empty((ns + m, 3), device=dev)
        cov3d = torch.zeros((ns + m, 6), device=dev)
        means[:ns] = s_means.detach()
        joint_ids, weights, avatar_of, n_avatars, n_joints = av_static
        dest = torch.arange(ns, ns + m, dtype=torch.int64, device=dev)
        av = Avatars(a_means.detach().contiguous(), a_ls.detach().contiguous(), a_q.detach().contiguous(),
                     joint_ids, weights, avatar_of, n_avatars, n_joints, dest=dest)
        deform(av, G.detach().contiguous(), means, cov3d)
        ls = torch.cat([s_ls.detach(), torch.zeros((m, 3), device=dev)])
        q = torch.cat([s_q.detach(), torch.tensor([[1.0, 0.0, 0.0, 0.0]], device=dev).expand(m, 4)]).contiguous()
        op = torch.cat([s_op.detach(), a_op.detach()]).contiguous()
        sh = torch.cat([s_sh.detach(), a_sh.detach()]).contiguous()
        g = Gaussians(means, ls, q, op, sh, cov3d)
        rgb, depth, T, nc = renderer.forward(g, cams)
        ctx.save = (g, av, G.detach().contiguous(), renderer, cams, ns, m, s_sh.dtype)
        return rgb, depth

    @staticmethod
    def backward(ctx, d_rgb, d_depth):
        g, av, G, r, cams, ns, m, shd = ctx.save
        V, H, W = r.batch.n_views, r.height, r.width
        if d_rgb is None:
            d_rgb = torch.zeros((V, 3, H, W), device=r.device)
        if d_depth is None:
            d_depth = torch.zeros((V, H, W), device=r.device)
        gr = r.backward(g, cams, d_rgb.float(), d_depth.float())
        ga = dict(means=torch.zeros((m, 3), device=r.device), log_scales=torch.zeros((m, 3), device=r.device),
                  quats=torch.zeros((m, 4), device=r.device), G=torch.zeros_like(G))
        deform_backward(av, G, gr["means"], gr["cov3d"], ga)
        return (gr["means"][:ns], gr["log_scales"][:ns], gr["quats"][:ns], gr["opacity_logits"][:ns],
                gr["sh"][:ns].to(shd), ga["means"], ga["log_scales"], ga["quats"], gr["opacity_logits"][ns:],
                gr["sh"][ns:].to(shd), ga["G"], None, None, None)
