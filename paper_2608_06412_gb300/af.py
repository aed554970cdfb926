"""Python binding of libaf (include/af.h): argument marshalling only.

Every step of the hot path runs in the CUDA library; this module turns torch
tensors and numpy arrays into pointers and af_* calls. PyTorch provides the
device memory and the streams. If the library is missing or no CUDA device
is present, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

UNSCORED, ACCESSIBLE, BLOCKED = 0, 1, 2
OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_CHECK = range(7)
KERNEL_TOOL, KERNEL_CORRIDOR = 0, 1
STATUS = {0: "AF_OK", 1: "AF_ERR_INVALID_ARG", 2: "AF_ERR_CAPACITY", 3: "AF_ERR_CUDA",
          4: "AF_ERR_TIMEOUT", 5: "AF_ERR_STATE"}

#: Every symbol include/af.h declares.
EXPORTS = ("af_version", "af_create", "af_destroy", "af_integrate_scan", "af_set_tool",
           "af_score", "af_frame_host", "af_sync_status", "af_get_stats", "af_block_count",
           "af_export_blocks", "af_kernel_offsets", "af_arm_offsets", "af_profile_enable",
           "af_profile_read", "af_integrate_scan_noalloc", "af_batch_create", "af_batch_destroy",
           "af_batch_tick", "af_batch_set_tuning", "af_batch_get_tuning", "af_soft_seed",
           "af_soft_clearance", "af_soft_clearance_adjoint", "af_soft_refine", "af_soft_best",
           "af_soft_start", "af_points_enable", "af_points_frame", "af_points_drain",
           "af_points_stats", "af_points_export", "af_integrate_scan_projective",
           "af_set_score_split", "af_probe_l2_read", "af_soft_set_view", "af_last_error")
NOALLOC_MAX_RETURNS = 65536
#: Kernel names in the order of af_profile's arrays.
KERNELS = ("k_alloc", "k_integrate", "k_bitview", "k_score", "k_views", "k_soft",
           "k_soft_adjoint", "k_soft_refine", "k_soft_seed", "k_soft_best")
#: Softmin temperature of the soft clearance (m).
TAU_S = 0.005


class AfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(C.Structure):
    _fields_ = [("voxel_size", C.c_float), ("truncation", C.c_float), ("r_c", C.c_float),
                ("cone_cos", C.c_float), ("range_min", C.c_float), ("range_max", C.c_float),
                ("clear_lo", C.c_float), ("clear_hi", C.c_float),
                ("cube_radius", C.c_int32), ("clear_samples", C.c_int32),
                ("w_min", C.c_uint32), ("w_cap", C.c_uint32), ("block_edge", C.c_uint32),
                ("domain_min", C.c_int32 * 3), ("domain_bricks", C.c_uint32 * 3),
                ("hash_capacity", C.c_uint32), ("pool_blocks", C.c_uint32),
                ("max_returns", C.c_uint32), ("max_points", C.c_uint32),
                ("clamp_signed", C.c_int32)]


class _Tool(C.Structure):
    _fields_ = [("radius", C.c_float), ("length", C.c_float), ("self_excl", C.c_float),
                ("corr_radius", C.c_float), ("corr_length", C.c_float),
                ("cos_theta_max", C.c_float), ("n_c", C.c_uint32),
                ("corridor_strict", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("scans", "returns_in", "returns_accepted",
                                          "blocks_allocated", "blocks_dirty_last",
                                          "points_in", "points_scored", "tests")]


class _Profile(C.Structure):
    _fields_ = [("launches", C.c_uint64 * 10), ("ms", C.c_double * 10)]


class _Refine(C.Structure):
    _fields_ = [("steps", C.c_uint32), ("lr_dir", C.c_float), ("lr_h", C.c_float),
                ("h_max", C.c_float)]


class _PointsConfig(C.Structure):
    _fields_ = [("capacity", C.c_uint32), ("k_nn", C.c_uint32), ("nn_radius", C.c_int32),
                ("max_views", C.c_uint32), ("view_min_dist", C.c_float), ("obs_dot", C.c_float),
                ("trig_tsdf", C.c_float), ("trig_move", C.c_float), ("budget", C.c_uint32),
                ("k_c", C.c_float), ("c_min", C.c_float), ("a_decay", C.c_float),
                ("a_recover", C.c_float), ("ca_min", C.c_float), ("c2f_stride", C.c_uint32),
                ("c2f_half", C.c_uint32), ("c2f_radius", C.c_float), ("trig_exact", C.c_int32),
                ("trig_radius", C.c_int32), ("trig_sample", C.c_uint32)]


class _BatchItem(C.Structure):
    _fields_ = [("d_xyz", C.c_void_p), ("n", C.c_uint32), ("pose", C.c_float * 16),
                ("d_pts", C.c_void_p), ("d_normals", C.c_void_p), ("m", C.c_uint32),
                ("d_label", C.c_void_p), ("d_best", C.c_void_p)]


class _Tuning(C.Structure):
    _fields_ = [("returns_per_tile", C.c_uint32), ("warps_per_cta", C.c_uint32),
                ("explored", C.c_uint32), ("done", C.c_uint32), ("ms", C.c_float * 9)]


_lib = None


def load(build: bool = True) -> C.CDLL:
    """Load libaf.so from the package directory (building it if stale); with
    the environment variable AF_CHECKED=1, the bounds-checked libaf_checked.so
    (same entry points; failed checks latch AF_ERR_CHECK)."""
    global _lib
    if _lib is None:
        if build:
            _build.build()
        path = _build.LIB_CHECKED if os.environ.get("AF_CHECKED") == "1" else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run build()")
        lib = C.CDLL(path)
        P, U32, I32, I64 = C.c_void_p, C.c_uint32, C.c_int32, C.c_int64
        sig = {
            "af_version": (C.c_char_p, []),
            "af_create": (C.c_int, [C.POINTER(_Config), C.POINTER(P)]),
            "af_destroy": (C.c_int, [P]),
            "af_integrate_scan": (C.c_int, [P, P, U32, P, P]),
            "af_integrate_scan_projective": (C.c_int, [P, P, U32, P, U32, P]),
            "af_set_score_split": (C.c_int, [P, C.c_int32]),
            "af_probe_l2_read": (C.c_int, [C.c_uint64, U32, U32, C.POINTER(C.c_double)]),
            "af_soft_set_view": (C.c_int, [P, C.c_int32]),
            "af_set_tool": (C.c_int, [P, C.POINTER(_Tool), P, U32]),
            "af_score": (C.c_int, [P, P, P, U32, P, P, P]),
            "af_frame_host": (C.c_int, [P, P, U32, P, P, P, U32, P, P, P]),
            "af_sync_status": (C.c_int, [P]),
            "af_get_stats": (C.c_int, [P, C.POINTER(_Stats)]),
            "af_block_count": (C.c_int, [P, C.POINTER(U32)]),
            "af_export_blocks": (C.c_int, [P, U32, P, P, P, P, C.POINTER(U32)]),
            "af_kernel_offsets": (C.c_int, [C.POINTER(_Tool), C.c_float, P, I32, P, I64,
                                            C.POINTER(I64)]),
            "af_arm_offsets": (C.c_int, [C.c_float, C.c_float, P, P]),
            "af_profile_enable": (C.c_int, [P, C.c_int]),
            "af_profile_read": (C.c_int, [P, C.POINTER(_Profile), C.c_int]),
            "af_integrate_scan_noalloc": (C.c_int, [C.POINTER(_Config), P, U32, P, P, P, P, P,
                                                    P]),
            "af_batch_create": (C.c_int, [P, U32, C.POINTER(P)]),
            "af_batch_destroy": (C.c_int, [P]),
            "af_batch_tick": (C.c_int, [P, P, P]),
            "af_batch_set_tuning": (C.c_int, [P, U32, U32]),
            "af_batch_get_tuning": (C.c_int, [P, C.POINTER(_Tuning)]),
            "af_soft_seed": (C.c_int, [P, P, U32, P, U32, P, P]),
            "af_soft_clearance": (C.c_int, [P, P, U32, P, P, P, P, C.c_uint64, C.c_float, P,
                                            P, P]),
            "af_soft_clearance_adjoint": (C.c_int, [P, P, U32, P, P, P, P, C.c_uint64,
                                                    C.c_float, P, P, P, P, P, P]),
            "af_soft_refine": (C.c_int, [P, P, U32, P, P, P, P, C.c_uint64, C.c_float,
                                         C.POINTER(_Refine), P, P, P]),
            "af_soft_best": (C.c_int, [P, P, C.c_uint64, U32, P, P, P, P, P]),
            "af_soft_start": (C.c_int, [P, P, P, U32, P, P]),
            "af_points_enable": (C.c_int, [P, C.POINTER(_PointsConfig)]),
            "af_points_frame": (C.c_int, [P, P, U32, P, P]),
            "af_points_drain": (C.c_int, [P, U32, P]),
            "af_points_stats": (C.c_int, [P, C.POINTER(U32), C.POINTER(U32)]),
            "af_points_export": (C.c_int, [P, U32, P, P, P, P, P, P, P, P, C.POINTER(U32)]),
            "af_last_error": (C.c_char_p, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


def _check(st: int, ctx=None):
    if st != 0:
        raise AfError(st, load().af_last_error(ctx).decode())


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dev_ptr(t, dtype, shape_tail=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor")
    if shape_tail is not None and tuple(t.shape[1:]) != shape_tail:
        raise TypeError(f"expected shape (n, {shape_tail})")
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


@dataclass
class MapConfig:
    """Map parameters (Sec. 3.2-3.6); the box is in bricks of 8^3 voxels."""
    voxel_size: float
    truncation: float
    r_c: float
    cube_radius: int
    clear_samples: int
    domain_min: tuple
    domain_bricks: tuple
    cone_cos: float = 0.95
    range_min: float = 0.1
    range_max: float = 40.0
    clear_lo: float = 1.0
    clear_hi: float = 2.25
    w_min: int = 3
    w_cap: int = 2000
    hash_capacity: int = 1 << 16
    pool_blocks: int = 1 << 15
    max_returns: int = 1 << 16
    max_points: int = 1 << 16
    clamp_signed: int = 0     # 1: contributions clamped to [-tau, tau] (Tab. 4 ablation)

    def _c(self) -> _Config:
        c = _Config()
        for k in ("voxel_size", "truncation", "r_c", "cone_cos", "range_min", "range_max",
                  "clear_lo", "clear_hi", "cube_radius", "clear_samples", "w_min", "w_cap",
                  "hash_capacity", "pool_blocks", "max_returns", "max_points", "clamp_signed"):
            setattr(c, k, getattr(self, k))
        c.block_edge = 8
        c.domain_min[:] = [int(x) for x in self.domain_min]
        c.domain_bricks[:] = [int(x) for x in self.domain_bricks]
        return c


@dataclass
class PointsConfig:
    """The stateful point layer (Sec. 3.4, 3.5); trig_tsdf is 2 v."""
    trig_tsdf: float
    capacity: int = 1 << 20
    k_nn: int = 10
    nn_radius: int = 3
    max_views: int = 8
    view_min_dist: float = 0.1
    obs_dot: float = 0.25
    trig_move: float = 0.1
    budget: int = 0xFFFFFFFF
    k_c: float = 5.0
    c_min: float = 0.2
    a_decay: float = 0.75
    a_recover: float = 0.15
    ca_min: float = 0.7
    # coarse-to-fine search over a ring-ordered direction table (Sec. 3.6);
    # for the 180-direction yaw ring: stride 10 (20 deg), half 12 (+-24 deg)
    c2f_stride: int = 0
    c2f_half: int = 0
    c2f_radius: float = 0.3
    # neighbourhood trigger: 1 = a changed voxel within trig_radius voxels
    # (r_u = 3v) among trig_sample changed voxels drawn per frame (0: all);
    # 0 = the brick rule (a touched brick next to the point's), a superset
    trig_exact: int = 1
    trig_radius: int = 3
    trig_sample: int = 256

    def _c(self) -> _PointsConfig:
        c = _PointsConfig()
        for k, _ in _PointsConfig._fields_:
            setattr(c, k, getattr(self, k))
        return c


@dataclass
class ToolConfig:
    """Cylinder tool with a coaxial approach corridor (Sec. 3.4)."""
    radius: float
    length: float
    self_excl: float
    corr_radius: float
    corr_length: float
    cos_theta_max: float = 0.0
    n_c: int = 5
    strict: int = 0

    def _c(self) -> _Tool:
        t = _Tool()
        for k in ("radius", "length", "self_excl", "corr_radius", "corr_length",
                  "cos_theta_max", "n_c"):
            setattr(t, k, getattr(self, k))
        t.corridor_strict = self.strict
        return t


class Map:
    """An accessibility-field map on the current CUDA device (af_create)."""

    def __init__(self, cfg: MapConfig):
        self.cfg = cfg
        self._lib = load()
        self._cc = cfg._c()
        h = C.c_void_p()
        _check(self._lib.af_create(C.byref(self._cc), C.byref(h)))
        self._h = h
        self.G = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.af_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate_scan(self, xyz, pose, stream=None):
        """af_integrate_scan: xyz is an (n, 3) float32 CUDA tensor (sensor frame),
        pose a 4x4 world_from_sensor matrix."""
        import torch
        n = int(xyz.shape[0])
        p = _dev_ptr(xyz, torch.float32, (3,)) if n else C.c_void_p(0)
        pose = np.ascontiguousarray(pose, np.float32).reshape(16)
        _check(self._lib.af_integrate_scan(self._h, p, n, _np_ptr(pose), _stream_ptr(stream)),
               self._h)

    def integrate_scan_projective(self, xyz, pose, bins: int = 812, stream=None):
        """af_integrate_scan_projective: the projective ablation of Tab. 3 over
        a bins x bins octahedral range image."""
        import torch
        n = int(xyz.shape[0])
        p = _dev_ptr(xyz, torch.float32, (3,)) if n else C.c_void_p(0)
        pose = np.ascontiguousarray(pose, np.float32).reshape(16)
        _check(self._lib.af_integrate_scan_projective(self._h, p, n, _np_ptr(pose), int(bins),
                                                      _stream_ptr(stream)), self._h)

    def set_score_split(self, budget: int):
        """af_set_score_split: -1 single pass; otherwise hand a point's directions
        beyond `budget` searched ones to per-direction warps (same results)."""
        _check(self._lib.af_set_score_split(self._h, int(budget)), self._h)

    def set_tool(self, tool: ToolConfig, dirs: np.ndarray):
        """af_set_tool: rasterise the tool/corridor kernels for G directions."""
        dirs = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
        self._tc = tool._c()
        _check(self._lib.af_set_tool(self._h, C.byref(self._tc), _np_ptr(dirs), len(dirs)),
               self._h)
        self.G = len(dirs)

    def score(self, pts, normals, label=None, best=None, stream=None):
        """af_score: returns (label uint8, best int16) CUDA tensors."""
        import torch
        m = int(pts.shape[0])
        if label is None:
            label = torch.empty(m, dtype=torch.uint8, device=pts.device)
        if best is None:
            best = torch.empty(m, dtype=torch.int16, device=pts.device)
        if m:
            _check(self._lib.af_score(self._h, _dev_ptr(pts, torch.float32, (3,)),
                                      _dev_ptr(normals, torch.float32, (3,)), m,
                                      _dev_ptr(label, torch.uint8), _dev_ptr(best, torch.int16),
                                      _stream_ptr(stream)), self._h)
        return label, best

    def frame_host(self, xyz: np.ndarray, pose, pts: np.ndarray, normals: np.ndarray,
                   label: np.ndarray, best: np.ndarray, stream=None):
        """af_frame_host: one frame from (ideally page-locked) host arrays."""
        pose = np.ascontiguousarray(pose, np.float32).reshape(16)
        _check(self._lib.af_frame_host(self._h, _np_ptr(xyz), len(xyz), _np_ptr(pose),
                                       _np_ptr(pts), _np_ptr(normals), len(pts),
                                       _np_ptr(label), _np_ptr(best), _stream_ptr(stream)),
               self._h)

    def sync_status(self) -> int:
        return int(self._lib.af_sync_status(self._h))

    def stats(self) -> dict:
        s = _Stats()
        _check(self._lib.af_get_stats(self._h, C.byref(s)), self._h)
        return {k: int(getattr(s, k)) for k, _ in _Stats._fields_}

    def profile(self, enable: bool = True):
        """Bracket every launch with CUDA events on its stream (af_profile_enable)."""
        _check(self._lib.af_profile_enable(self._h, int(enable)), self._h)

    def profile_read(self, reset: bool = True) -> dict:
        """{kernel: (launches, total ms)} since the last reset (af_profile_read)."""
        p = _Profile()
        _check(self._lib.af_profile_read(self._h, C.byref(p), int(reset)), self._h)
        return {k: (int(p.launches[i]), float(p.ms[i])) for i, k in enumerate(KERNELS)}

    def block_count(self) -> int:
        n = C.c_uint32()
        _check(self._lib.af_block_count(self._h, C.byref(n)), self._h)
        return int(n.value)

    def export_blocks(self, cap: int | None = None) -> dict:
        """Allocated bricks (all, or the first `cap` in pool order): absolute
        brick keys and per-voxel S, w, flags."""
        n = self.block_count() if cap is None else min(cap, self.block_count())
        key = np.zeros((max(n, 1), 3), np.int32)
        S = np.zeros((max(n, 1), 512), np.int64)
        w = np.zeros((max(n, 1), 512), np.uint32)
        fl = np.zeros((max(n, 1), 512), np.uint8)
        out = C.c_uint32()
        _check(self._lib.af_export_blocks(self._h, n, _np_ptr(key), _np_ptr(S), _np_ptr(w),
                                          _np_ptr(fl), C.byref(out)), self._h)
        n = int(out.value)
        return dict(key=key[:n], S=S[:n], w=w[:n], flags=fl[:n])

    # ---- the stateful point layer ----

    def points_enable(self, cfg: "PointsConfig"):
        """af_points_enable."""
        self._pc = cfg._c()
        _check(self._lib.af_points_enable(self._h, C.byref(self._pc)), self._h)

    def points_frame(self, xyz, pose, stream=None):
        """af_points_frame: integrate a scan and update the point layer."""
        import torch
        n = int(xyz.shape[0])
        p = _dev_ptr(xyz, torch.float32, (3,)) if n else C.c_void_p(0)
        pose = np.ascontiguousarray(pose, np.float32).reshape(16)
        _check(self._lib.af_points_frame(self._h, p, n, _np_ptr(pose), _stream_ptr(stream)),
               self._h)

    def points_drain(self, max_evals: int, stream=None):
        """af_points_drain: evaluate up to max_evals queued points."""
        _check(self._lib.af_points_drain(self._h, max_evals, _stream_ptr(stream)), self._h)

    def points_stats(self) -> tuple:
        """(number of points, evaluations of the last frame or drain)."""
        n, e = C.c_uint32(), C.c_uint32()
        _check(self._lib.af_points_stats(self._h, C.byref(n), C.byref(e)), self._h)
        return int(n.value), int(e.value)

    def points_export(self) -> dict:
        """Every point in id order: ijk, normal, label, score, best, a, queued, nviews."""
        n, _ = self.points_stats()
        out = dict(ijk=np.zeros((n, 3), np.int32), normal=np.zeros((n, 3), np.float32),
                   label=np.zeros(n, np.uint8), score=np.zeros(n, np.int16),
                   best=np.zeros(n, np.int16), a=np.zeros(n, np.float32),
                   queued=np.zeros(n, np.uint8), nviews=np.zeros(n, np.int32))
        cnt = C.c_uint32()
        _check(self._lib.af_points_export(self._h, n, *(_np_ptr(out[k]) for k in
                                                        ("ijk", "normal", "label", "score", "best",
                                                         "a", "queued", "nviews")),
                                          C.byref(cnt)), self._h)
        return out

    # ---- the differentiable form ----

    def soft_seed(self, normals, table, out=None, stream=None):
        """af_soft_seed: (m*K, 3) base directions, the K rows of `table`
        (K x 3, around +z) rotated into each normal's tangent frame."""
        import torch
        m = int(normals.shape[0])
        table = np.ascontiguousarray(table, np.float32).reshape(-1, 3)
        u0 = out if out is not None else \
            torch.empty((m * len(table), 3), dtype=torch.float32, device=normals.device)
        _check(self._lib.af_soft_seed(self._h, _dev_ptr(normals, torch.float32, (3,)) if m
                                      else C.c_void_p(0), m, _np_ptr(table), len(table),
                                      _dev_ptr(u0, torch.float32, (3,)) if m else C.c_void_p(0),
                                      _stream_ptr(stream)), self._h)
        return u0

    def soft_set_view(self, mode: int):
        """af_soft_set_view: 0 automatic, 1 dense, 2 brick-sparse SDF view."""
        _check(self._lib.af_soft_set_view(self._h, int(mode)), self._h)

    def soft_start(self, label, best, out=None, stream=None):
        """af_soft_start: (m, 3) start directions of refinement -- the best
        direction of each ACCESSIBLE point of af_score's output, NaN for the
        others."""
        import torch
        m = int(label.shape[0])
        u0 = out if out is not None else \
            torch.empty((m, 3), dtype=torch.float32, device=label.device)
        z = C.c_void_p(0)
        _check(self._lib.af_soft_start(self._h, _dev_ptr(label, torch.uint8) if m else z,
                                       _dev_ptr(best, torch.int16) if m else z, m,
                                       _dev_ptr(u0, torch.float32, (3,)) if m else z,
                                       _stream_ptr(stream)), self._h)
        return u0

    def _pair_ptrs(self, pts, u0, alpha, beta, h, per_point):
        import torch
        n = int(u0.shape[0])
        if per_point < 1 or int(pts.shape[0]) * per_point < n:
            raise ValueError("need per_point >= 1 and a point for every pair")
        for t in (alpha, beta, h):
            if t.shape != (n,):
                raise ValueError("alpha, beta and h need one value per pair")
        if n == 0:
            return n, [C.c_void_p(0)] * 5
        return n, [_dev_ptr(pts, torch.float32, (3,)), _dev_ptr(u0, torch.float32, (3,)),
                   _dev_ptr(alpha, torch.float32), _dev_ptr(beta, torch.float32),
                   _dev_ptr(h, torch.float32)]

    def soft_clearance_raw(self, pts, u0, alpha, beta, h, per_point, tau_s=TAU_S, out=None,
                           cmin=None, stream=None):
        """af_soft_clearance: C of every pair (no autograd); `cmin`, if
        given, receives the hard clearance."""
        import torch
        n, ptr = self._pair_ptrs(pts, u0, alpha, beta, h, per_point)
        c = torch.empty(n, dtype=torch.float32, device=u0.device) if out is None else out
        _check(self._lib.af_soft_clearance(self._h, ptr[0], per_point, *ptr[1:], n, tau_s,
                                           _dev_ptr(c, torch.float32) if n else C.c_void_p(0),
                                           _dev_ptr(cmin, torch.float32) if (cmin is not None
                                                                            and n)
                                           else C.c_void_p(0), _stream_ptr(stream)), self._h)
        return c

    def soft_clearance_adjoint(self, pts, u0, alpha, beta, h, per_point, tau_s=TAU_S,
                               grad_c=None, stream=None):
        """af_soft_clearance_adjoint: (C, g dC/dalpha, g dC/dbeta, g dC/dh)."""
        import torch
        n, ptr = self._pair_ptrs(pts, u0, alpha, beta, h, per_point)
        out = [torch.empty(n, dtype=torch.float32, device=u0.device) for _ in range(4)]
        op = [_dev_ptr(t, torch.float32) if n else C.c_void_p(0) for t in out]
        gp = _dev_ptr(grad_c, torch.float32) if (grad_c is not None and n) else C.c_void_p(0)
        _check(self._lib.af_soft_clearance_adjoint(self._h, ptr[0], per_point, *ptr[1:], n,
                                                   tau_s, gp, *op, _stream_ptr(stream)),
               self._h)
        return tuple(out)

    def soft_clearance(self, pts, u0, alpha, beta, h, per_point, tau_s=TAU_S):
        """C of every pair, differentiable in alpha, beta and h (SoftClearance)."""
        return SoftClearance.apply(self, pts, u0, alpha, beta, h, per_point, tau_s)

    def soft_refine(self, pts, u0, alpha, beta, h, per_point=1, steps=20, lr_dir=0.05,
                    lr_h=0.005, h_max=0.05, tau_s=TAU_S, out=None, stream=None):
        """af_soft_refine: `steps` ascent steps on every pair in one launch;
        alpha, beta, h are updated in place. Returns (C, hard clearance)."""
        import torch
        n, ptr = self._pair_ptrs(pts, u0, alpha, beta, h, per_point)
        R = _Refine(steps, lr_dir, lr_h, h_max)
        c, cmin = out if out is not None else \
            (torch.empty(n, dtype=torch.float32, device=u0.device),
             torch.empty(n, dtype=torch.float32, device=u0.device))
        op = [_dev_ptr(t, torch.float32) if n else C.c_void_p(0) for t in (c, cmin)]
        _check(self._lib.af_soft_refine(self._h, ptr[0], per_point, *ptr[1:], n, tau_s,
                                        C.byref(R), *op, _stream_ptr(stream)), self._h)
        return c, cmin

    def soft_best(self, c, per_point, u0=None, out=None, stream=None):
        """af_soft_best: per point (index of its largest C, that C, and --
        with u0 -- that pair's base direction)."""
        import torch
        n = int(c.shape[0])
        npts = (n + per_point - 1) // per_point
        if out is not None:
            bk, bc, bu = out
        else:
            bk = torch.empty(npts, dtype=torch.int32, device=c.device)
            bc = torch.empty(npts, dtype=torch.float32, device=c.device)
            bu = torch.empty((npts, 3), dtype=torch.float32, device=c.device) \
                if u0 is not None else None
        z = C.c_void_p(0)
        _check(self._lib.af_soft_best(self._h, _dev_ptr(c, torch.float32) if n else z, n,
                                      per_point, _dev_ptr(u0, torch.float32, (3,))
                                      if (u0 is not None and n) else z,
                                      _dev_ptr(bk, torch.int32) if npts else z,
                                      _dev_ptr(bc, torch.float32) if npts else z,
                                      _dev_ptr(bu, torch.float32, (3,)) if (bu is not None and
                                                                           npts) else z,
                                      _stream_ptr(stream)), self._h)
        return (bk, bc, bu) if u0 is not None else (bk, bc)


def _soft_function():
    import torch

    class SoftClearance(torch.autograd.Function):
        """C = soft clearance of (point, direction) pairs; backward runs the
        adjoint kernel, which recomputes every SDF sample from the map (only
        the inputs are saved)."""

        @staticmethod
        def forward(ctx, m, pts, u0, alpha, beta, h, per_point, tau_s):
            ctx.save_for_backward(pts, u0, alpha, beta, h)
            ctx.m, ctx.per_point, ctx.tau_s = m, per_point, tau_s
            return m.soft_clearance_raw(pts, u0, alpha.detach(), beta.detach(), h.detach(),
                                        per_point, tau_s)

        @staticmethod
        def backward(ctx, grad_c):
            pts, u0, alpha, beta, h = ctx.saved_tensors
            _, ga, gb, gh = ctx.m.soft_clearance_adjoint(
                pts, u0, alpha.detach(), beta.detach(), h.detach(), ctx.per_point, ctx.tau_s,
                grad_c.contiguous())
            return (None, None, None, ga if ctx.needs_input_grad[3] else None,
                    gb if ctx.needs_input_grad[4] else None,
                    gh if ctx.needs_input_grad[5] else None, None, None)

    return SoftClearance


class _LazySoft:
    _fn = None

    def apply(self, *args):
        if _LazySoft._fn is None:
            _LazySoft._fn = _soft_function()
        return _LazySoft._fn.apply(*args)


#: torch.autograd.Function of the soft clearance: SoftClearance.apply(map,
#: pts, u0, alpha, beta, h, per_point, tau_s).
SoftClearance = _LazySoft()


def export_voxels(blocks: dict) -> dict:
    """Flatten exported bricks to the voxels that carry state (w > 0 or
    cleared), sorted by (z, y, x): ijk, S, w, cleared, occ, known."""
    key, S, w, fl = blocks["key"], blocks["S"], blocks["w"], blocks["flags"]
    l = np.arange(512)
    loc = np.stack([l & 7, (l >> 3) & 7, l >> 6], 1)
    ijk = (key[:, None, :] * 8 + loc[None]).reshape(-1, 3)
    S, w, fl = S.reshape(-1), w.reshape(-1), fl.reshape(-1)
    keep = (w > 0) | ((fl & 1) != 0)
    ijk, S, w, fl = ijk[keep], S[keep], w[keep], fl[keep]
    order = np.lexsort((ijk[:, 0], ijk[:, 1], ijk[:, 2]))
    return dict(ijk=ijk[order].astype(np.int32), S=S[order], w=w[order],
                cleared=(fl[order] & 1).astype(np.uint8),
                occ=((fl[order] >> 1) & 1).astype(np.uint8),
                known=((fl[order] >> 2) & 1).astype(np.uint8))


def kernel_offsets(tool: ToolConfig, v: float, u, which: int) -> np.ndarray:
    """Host-only af_kernel_offsets, sorted z-major."""
    lib = load()
    tc = tool._c()
    u = np.ascontiguousarray(u, np.float32).reshape(3)
    cnt = C.c_int64()
    _check(lib.af_kernel_offsets(C.byref(tc), v, _np_ptr(u), which, None, 0, C.byref(cnt)))
    out = np.zeros((max(cnt.value, 1), 3), np.int32)
    _check(lib.af_kernel_offsets(C.byref(tc), v, _np_ptr(u), which, _np_ptr(out), cnt.value,
                                 C.byref(cnt)))
    out = out[:cnt.value]
    return out[np.lexsort((out[:, 0], out[:, 1], out[:, 2]))]


def probe_l2_read(nbytes: int = 32 << 20, reps: int = 40, launches: int = 20) -> float:
    """af_probe_l2_read: the L2 read bandwidth (GB/s) of the current device,
    measured by the library's own kernel on an L2-resident working set."""
    lib = load()
    out = C.c_double()
    _check(lib.af_probe_l2_read(nbytes, reps, launches, C.byref(out)))
    return float(out.value)


def arm_offsets(v: float, tau: float, u) -> np.ndarray:
    lib = load()
    u = np.ascontiguousarray(u, np.float32).reshape(3)
    out = np.zeros((3, 3), np.int32)
    _check(lib.af_arm_offsets(v, tau, _np_ptr(u), _np_ptr(out)))
    return out


def integrate_scan_noalloc(cfg: MapConfig, xyz, pose, box_min, box_dim, vox, flags,
                           stream=None):
    """af_integrate_scan_noalloc: add one scan to a caller-owned dense voxel box
    (vox: int64 CUDA tensor of (S << 20) | w words, flags: uint8 CUDA tensor;
    both box_dim[0] * box_dim[1] * box_dim[2] long). The library allocates
    nothing for this call, for callers that cannot allocate device memory."""
    import torch
    lib = load()
    cc = cfg._c()
    n = int(xyz.shape[0])
    p = _dev_ptr(xyz, torch.float32, (3,)) if n else C.c_void_p(0)
    pose = np.ascontiguousarray(pose, np.float32).reshape(16)
    bmin = np.ascontiguousarray(box_min, np.int32).reshape(3)
    bdim = np.ascontiguousarray(box_dim, np.uint32).reshape(3)
    count = int(np.prod(bdim.astype(np.int64)))
    if vox.numel() != count or flags.numel() != count:
        raise ValueError("vox and flags must hold box_dim[0] * box_dim[1] * box_dim[2] voxels")
    _check(lib.af_integrate_scan_noalloc(C.byref(cc), p, n, _np_ptr(pose), _np_ptr(bmin),
                                         _np_ptr(bdim), _dev_ptr(vox, torch.int64),
                                         _dev_ptr(flags, torch.uint8), _stream_ptr(stream)))


class Batch:
    """Many maps ticked together (af_batch_*): each tick integrates every
    scene's scan and scores its points, as one CUDA graph launch."""

    def __init__(self, maps):
        self.maps = list(maps)
        self._lib = load()
        arr = (C.c_void_p * len(self.maps))(*[m._h.value for m in self.maps])
        h = C.c_void_p()
        _check(self._lib.af_batch_create(arr, len(self.maps), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.af_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tick(self, items, stream=None):
        """items[s] = (xyz, pose, pts, normals, label, best) for scene s: CUDA
        tensors as for Map.integrate_scan / Map.score (pts may hold 0 rows).
        The tensors must stay alive until the tick has run."""
        import torch
        arr = (_BatchItem * len(self.maps))()
        for s, (xyz, pose, pts, nrm, lab, best) in enumerate(items):
            it = arr[s]
            it.n = int(xyz.shape[0])
            it.d_xyz = _dev_ptr(xyz, torch.float32, (3,)).value if it.n else None
            it.pose[:] = [float(x) for x in np.asarray(pose, np.float32).reshape(16)]
            it.m = int(pts.shape[0])
            if it.m:
                it.d_pts = _dev_ptr(pts, torch.float32, (3,)).value
                it.d_normals = _dev_ptr(nrm, torch.float32, (3,)).value
                it.d_label = _dev_ptr(lab, torch.uint8).value
                it.d_best = _dev_ptr(best, torch.int16).value
        _check(self._lib.af_batch_tick(self._h, arr, _stream_ptr(stream)))

    def set_tuning(self, returns_per_tile: int, warps_per_cta: int):
        _check(self._lib.af_batch_set_tuning(self._h, returns_per_tile, warps_per_cta))

    def tuning(self) -> dict:
        t = _Tuning()
        _check(self._lib.af_batch_get_tuning(self._h, C.byref(t)))
        return dict(returns_per_tile=t.returns_per_tile, warps_per_cta=t.warps_per_cta,
                    explored=t.explored, done=bool(t.done), ms=list(t.ms))
