"""Plain CPU oracle of the Accessibility Field hot path (ctypes over af_oracle.c).

TEST INFRASTRUCTURE. The oracle is the correctness reference for the CUDA
path: scan-centric TSDF integration with positive clamping (Sec. 3.2), the
ray-cleared free band (Sec. 3.4), the weight cap (Sec. 3.6), the occupied /
known view, and accessibility scoring against tool and corridor kernels
(Sec. 3.4, 3.5). Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it. It imports nothing from the
product package and the product imports nothing from here.

All arithmetic lives in ``af_oracle.c``; this module only marshals arrays.
Parity status of each function is recorded in the module docstrings of the
tests that pin it (``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, f) for f in ("af_oracle.c", "af_oracle_points.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

UNSCORED, ACCESSIBLE, BLOCKED = 0, 1, 2
KERNEL_TOOL, KERNEL_CORRIDOR = 0, 1


def build(force: bool = False) -> str:
    """Compile af_oracle.c with strict IEEE single-precision semantics."""
    deps = _SRCS + [os.path.join(_HERE, "af_oracle.h")]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(C.Structure):
    _fields_ = [("v", C.c_float), ("tau", C.c_float), ("r_c", C.c_float),
                ("cone_cos", C.c_float), ("range_min", C.c_float),
                ("range_max", C.c_float), ("clear_lo", C.c_float),
                ("clear_hi", C.c_float), ("cube_radius", C.c_int32),
                ("clear_samples", C.c_int32), ("w_min", C.c_uint32),
                ("w_cap", C.c_uint32), ("dom_min", C.c_int32 * 3),
                ("dom_size", C.c_int32 * 3), ("clamp_signed", C.c_int32)]


class _Tool(C.Structure):
    _fields_ = [("radius", C.c_float), ("length", C.c_float),
                ("self_excl", C.c_float), ("corr_radius", C.c_float),
                ("corr_length", C.c_float), ("cos_theta_max", C.c_float),
                ("n_c", C.c_uint32), ("strict", C.c_int32)]


_lib = None


class _PtsConfig(C.Structure):
    _fields_ = [("k_nn", C.c_uint32), ("nn_radius", C.c_int32), ("max_views", C.c_uint32),
                ("view_min_dist", C.c_float), ("obs_dot", C.c_float), ("trig_tsdf", C.c_float),
                ("trig_move", C.c_float), ("budget", C.c_uint32), ("k_c", C.c_float),
                ("c_min", C.c_float), ("a_decay", C.c_float), ("a_recover", C.c_float),
                ("ca_min", C.c_float), ("c2f_stride", C.c_uint32), ("c2f_half", C.c_uint32),
                ("c2f_radius", C.c_float), ("trig_exact", C.c_int32), ("trig_radius", C.c_int32),
                ("trig_sample", C.c_uint32)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.or_map_new.restype = P
        lib.or_map_new.argtypes = [C.POINTER(_Config)]
        lib.or_map_free.argtypes = [P]
        lib.or_integrate.restype = C.c_int64
        lib.or_integrate.argtypes = [P, P, C.c_int64, P]
        lib.or_integrate_projective.restype = C.c_int64
        lib.or_integrate_projective.argtypes = [P, P, C.c_int64, P, C.c_int32]
        lib.or_octa_bin.restype = C.c_int32
        lib.or_octa_bin.argtypes = [P, C.c_int32]
        lib.or_get_voxel.restype = C.c_int
        lib.or_get_voxel.argtypes = [P, C.c_int32, C.c_int32, C.c_int32,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_uint32),
                                     C.POINTER(C.c_int32)]
        lib.or_set_voxel.argtypes = [P, C.c_int32, C.c_int32, C.c_int32,
                                     C.c_int64, C.c_uint32, C.c_int32]
        lib.or_set_voxels.argtypes = [P, C.c_int64, P, P, P, P]
        lib.or_voxel_count.restype = C.c_int64
        lib.or_voxel_count.argtypes = [P]
        lib.or_export.argtypes = [P, P, P, P, P, P, P]
        lib.or_occ.restype = C.c_int
        lib.or_occ.argtypes = [P, C.c_int32, C.c_int32, C.c_int32]
        lib.or_known.restype = C.c_int
        lib.or_known.argtypes = [P, C.c_int32, C.c_int32, C.c_int32]
        lib.or_kernel_offsets.restype = C.c_int64
        lib.or_kernel_offsets.argtypes = [C.POINTER(_Tool), C.c_float, P, C.c_int, P,
                                          C.c_int64]
        lib.or_arm_offsets.argtypes = [C.c_float, C.c_float, P, P]
        lib.or_score.argtypes = [P, C.POINTER(_Tool), P, C.c_int32, P, P, C.c_int64,
                                 P, P, P]
        lib.or_tables_new.restype = P
        lib.or_tables_new.argtypes = [C.POINTER(_Tool), C.c_float, C.c_float, P, C.c_int32]
        lib.or_tables_free.argtypes = [P]
        lib.or_score_tables.argtypes = [P, P, P, P, C.c_int64, P, P, P]
        lib.or_soft_clearance.argtypes = [P, C.POINTER(_Tool), P, C.c_uint32, P, P, P, P,
                                          C.c_int64, C.c_double, C.c_int, P, P, P, P, P]
        lib.or_soft_seed.argtypes = [P, C.c_int64, P, C.c_int32, P]
        lib.or_integrate2.restype = C.c_int64
        lib.or_integrate2.argtypes = [P, P, C.c_int64, P, P]
        lib.or_pts_new.restype = P
        lib.or_pts_new.argtypes = [P, C.POINTER(_PtsConfig), C.POINTER(_Tool), P, C.c_int32]
        lib.or_pts_free.argtypes = [P]
        lib.or_pts_frame.restype = C.c_int64
        lib.or_pts_frame.argtypes = [P, P, P, C.c_int64, P]
        lib.or_pts_drain.restype = C.c_int64
        lib.or_pts_drain.argtypes = [P, P, C.c_int64]
        lib.or_pts_count.restype = C.c_int64
        lib.or_pts_count.argtypes = [P]
        lib.or_pts_export.argtypes = [P, P, P, P, P, P, P, P, P]
        lib.or_jacobi3.argtypes = [P, C.c_int, P, P]
        lib.or_mix64.restype = C.c_uint64
        lib.or_mix64.argtypes = [C.c_uint64]
        lib.or_pts_state_step.argtypes = [C.POINTER(_PtsConfig), C.c_int32, C.c_int32, C.c_int32,
                                          C.c_float, P, P, P, P]
        lib.or_soft_refine.argtypes = [P, C.POINTER(_Tool), P, C.c_uint32, P, P, P, P,
                                       C.c_int64, C.c_double, C.c_int, C.c_float, C.c_float,
                                       C.c_float, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Config:
    """Map parameters (Sec. 3.2-3.6); voxel box = [dom_min, dom_min + dom_size)."""
    v: float
    tau: float
    r_c: float
    cube_radius: int
    clear_samples: int
    dom_min: tuple
    dom_size: tuple
    cone_cos: float = 0.95
    range_min: float = 0.1
    range_max: float = 40.0
    clear_lo: float = 1.0
    clear_hi: float = 2.25
    w_min: int = 3
    w_cap: int = 2000
    clamp_signed: int = 0   # 1: contributions clamped to [-tau, tau] (Tab. 4 ablation)

    def _c(self) -> _Config:
        c = _Config()
        for k in ("v", "tau", "r_c", "cone_cos", "range_min", "range_max",
                  "clear_lo", "clear_hi", "cube_radius", "clear_samples",
                  "w_min", "w_cap", "clamp_signed"):
            setattr(c, k, getattr(self, k))
        c.dom_min[:] = [int(x) for x in self.dom_min]
        c.dom_size[:] = [int(x) for x in self.dom_size]
        return c


@dataclass
class Tool:
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
                  "cos_theta_max", "n_c", "strict"):
            setattr(t, k, getattr(self, k))
        return t


class Map:
    """Voxel map of the oracle: S (units of 2^-20 m), w, cleared per voxel."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self._cc = cfg._c()
        self._lib = _load()
        self._h = self._lib.or_map_new(C.byref(self._cc))

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_map_free(self._h)
            self._h = None

    def integrate(self, pts: np.ndarray, pose: np.ndarray | None = None) -> int:
        pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
        pose = np.eye(4, dtype=np.float32) if pose is None else \
            np.ascontiguousarray(pose, dtype=np.float32).reshape(4, 4)
        return int(self._lib.or_integrate(self._h, _ptr(pts), len(pts), _ptr(pose)))

    def integrate_projective(self, pts: np.ndarray, pose: np.ndarray | None = None,
                             bins: int = 812) -> int:
        """Projective integration (the ablation of Tab. 3) over a bins x bins
        octahedral range image."""
        pts = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
        pose = np.eye(4, dtype=np.float32) if pose is None else \
            np.ascontiguousarray(pose, dtype=np.float32).reshape(4, 4)
        return int(self._lib.or_integrate_projective(self._h, _ptr(pts), len(pts), _ptr(pose),
                                                     int(bins)))

    def voxel(self, i: int, j: int, k: int):
        S, w, cl = C.c_int64(), C.c_uint32(), C.c_int32()
        self._lib.or_get_voxel(self._h, i, j, k, C.byref(S), C.byref(w), C.byref(cl))
        return int(S.value), int(w.value), int(cl.value)

    def set_voxel(self, i: int, j: int, k: int, S: int, w: int, cleared: int = 0):
        self._lib.or_set_voxel(self._h, i, j, k, S, w, cleared)

    def set_voxels(self, ijk: np.ndarray, S: np.ndarray, w: np.ndarray,
                   cleared: np.ndarray | None = None):
        ijk = np.ascontiguousarray(ijk, np.int32).reshape(-1, 3)
        n = len(ijk)
        S = np.ascontiguousarray(np.broadcast_to(S, (n,)), np.int64)
        w = np.ascontiguousarray(np.broadcast_to(w, (n,)), np.uint32)
        cl = np.zeros(n, np.uint8) if cleared is None else \
            np.ascontiguousarray(np.broadcast_to(cleared, (n,)), np.uint8)
        self._lib.or_set_voxels(self._h, n, _ptr(ijk), _ptr(S), _ptr(w), _ptr(cl))

    def occ(self, i: int, j: int, k: int) -> int:
        return int(self._lib.or_occ(self._h, i, j, k))

    def known(self, i: int, j: int, k: int) -> int:
        return int(self._lib.or_known(self._h, i, j, k))

    def __len__(self):
        return int(self._lib.or_voxel_count(self._h))

    def export(self) -> dict:
        """All stored voxels, sorted by (z, y, x)."""
        n = len(self)
        ijk = np.zeros((n, 3), np.int32)
        S = np.zeros(n, np.int64)
        w = np.zeros(n, np.uint32)
        cl = np.zeros(n, np.uint8)
        occ = np.zeros(n, np.uint8)
        kn = np.zeros(n, np.uint8)
        self._lib.or_export(self._h, _ptr(ijk), _ptr(S), _ptr(w), _ptr(cl), _ptr(occ),
                            _ptr(kn))
        order = np.lexsort((ijk[:, 0], ijk[:, 1], ijk[:, 2]))
        return dict(ijk=ijk[order], S=S[order], w=w[order], cleared=cl[order],
                    occ=occ[order], known=kn[order])

    def score(self, tool: Tool, dirs: np.ndarray, pts: np.ndarray, normals: np.ndarray,
              dir_scores: bool = False):
        dirs = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        normals = np.ascontiguousarray(normals, np.float32).reshape(-1, 3)
        m, G = len(pts), len(dirs)
        label = np.zeros(m, np.uint8)
        best = np.zeros(m, np.int16)
        ds = np.zeros((m, G), np.int32) if dir_scores else None
        tc = tool._c()
        self._lib.or_score(self._h, C.byref(tc), _ptr(dirs), G, _ptr(pts), _ptr(normals), m,
                           _ptr(label), _ptr(best), _ptr(ds) if ds is not None else None)
        return (label, best, ds) if dir_scores else (label, best)

    def score_tables(self, tables: "ScoreTables", pts: np.ndarray, normals: np.ndarray,
                     dir_scores: bool = False):
        """Map.score with kernel tables built once (or_score_tables)."""
        if (tables.cfg.v, tables.cfg.tau) != (self.cfg.v, self.cfg.tau):
            raise ValueError("tables were built for another voxel size or truncation")
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        normals = np.ascontiguousarray(normals, np.float32).reshape(-1, 3)
        m, G = len(pts), len(tables.dirs)
        label = np.zeros(m, np.uint8)
        best = np.zeros(m, np.int16)
        ds = np.zeros((m, G), np.int32) if dir_scores else None
        self._lib.or_score_tables(self._h, tables._h, _ptr(pts), _ptr(normals), m, _ptr(label),
                                  _ptr(best), _ptr(ds) if ds is not None else None)
        return (label, best, ds) if dir_scores else (label, best)

    def soft_clearance(self, tool: Tool, pts: np.ndarray, per_point: int, u0: np.ndarray,
                       alpha: np.ndarray, beta: np.ndarray, h: np.ndarray,
                       tau_s: float = 0.005, fp32_cells: bool = True):
        """Soft clearance C, dC/d(alpha, beta, h) (n x 3) and the hard
        clearance min_j phi_j of every pair, float64. Pair i belongs to point
        i // per_point."""
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        u0 = np.ascontiguousarray(u0, np.float32).reshape(-1, 3)
        n = len(u0)
        a, b, hh = (np.ascontiguousarray(x, np.float32).reshape(n) for x in (alpha, beta, h))
        if per_point < 1 or len(pts) * per_point < n:
            raise ValueError("need per_point >= 1 and a point for every pair")
        c, cmin = np.zeros(n), np.zeros(n)
        ga, gb, gh = np.zeros(n), np.zeros(n), np.zeros(n)
        tc = tool._c()
        self._lib.or_soft_clearance(self._h, C.byref(tc), _ptr(pts), per_point, _ptr(u0),
                                    _ptr(a), _ptr(b), _ptr(hh), n, tau_s, int(fp32_cells),
                                    _ptr(c), _ptr(ga), _ptr(gb), _ptr(gh), _ptr(cmin))
        self.last_cmin = cmin
        return c, np.stack([ga, gb, gh], 1)

    def soft_refine(self, tool: Tool, pts: np.ndarray, per_point: int, u0: np.ndarray,
                    alpha: np.ndarray, beta: np.ndarray, h: np.ndarray, steps: int,
                    lr_dir: float, lr_h: float, h_max: float, tau_s: float = 0.005):
        """(alpha, beta, h, C, hard clearance) after `steps` ascent steps."""
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        u0 = np.ascontiguousarray(u0, np.float32).reshape(-1, 3)
        n = len(u0)
        a, b, hh = (np.array(x, np.float32).reshape(n) for x in (alpha, beta, h))
        if per_point < 1 or len(pts) * per_point < n:
            raise ValueError("need per_point >= 1 and a point for every pair")
        c, cmin = np.zeros(n), np.zeros(n)
        tc = tool._c()
        self._lib.or_soft_refine(self._h, C.byref(tc), _ptr(pts), per_point, _ptr(u0), _ptr(a),
                                 _ptr(b), _ptr(hh), n, tau_s, steps, lr_dir, lr_h, h_max,
                                 _ptr(c), _ptr(cmin))
        return a, b, hh, c, cmin


def soft_seed(normals: np.ndarray, table: np.ndarray) -> np.ndarray:
    """Base directions (P*K, 3): the K table directions around each normal."""
    lib = _load()
    normals = np.ascontiguousarray(normals, np.float32).reshape(-1, 3)
    table = np.ascontiguousarray(table, np.float32).reshape(-1, 3)
    out = np.zeros((len(normals) * len(table), 3), np.float32)
    lib.or_soft_seed(_ptr(normals), len(normals), _ptr(table), len(table), _ptr(out))
    return out

def kernel_offsets(tool: Tool, v: float, u, which: int) -> np.ndarray:
    """Voxel offsets of the tool (which=0) or corridor (which=1) kernel of u."""
    lib = _load()
    u = np.ascontiguousarray(u, np.float32).reshape(3)
    tc = tool._c()
    n = lib.or_kernel_offsets(C.byref(tc), v, _ptr(u), which, None, 0)
    out = np.zeros((max(n, 1), 3), np.int32)
    lib.or_kernel_offsets(C.byref(tc), v, _ptr(u), which, _ptr(out), n)
    return out[:n]


def arm_offsets(v: float, tau: float, u) -> np.ndarray:
    """The three arm-path sample offsets (rows: 0.6, 1.25, 2.25 tau)."""
    lib = _load()
    u = np.ascontiguousarray(u, np.float32).reshape(3)
    out = np.zeros((3, 3), np.int32)
    lib.or_arm_offsets(C.c_float(v), C.c_float(tau), _ptr(u), _ptr(out))
    return out


class ScoreTables:
    """The kernel tables of one tool over a direction set, built once for a
    voxel size and truncation (Sec. 3.6: precomputed at initialisation)."""

    def __init__(self, cfg: Config, tool: Tool, dirs: np.ndarray):
        self._lib = _load()
        self.cfg = cfg
        self.dirs = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
        self._tc = tool._c()
        self._h = self._lib.or_tables_new(C.byref(self._tc), cfg.v, cfg.tau, _ptr(self.dirs),
                                          len(self.dirs))

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_tables_free(self._h)
            self._h = None


@dataclass
class PointsConfig:
    """The stateful layer's parameters (Sec. 3.4, 3.5); trig_tsdf is 2v."""
    trig_tsdf: float
    k_nn: int = 10
    nn_radius: int = 3
    max_views: int = 8
    view_min_dist: float = 0.1
    obs_dot: float = 0.25
    trig_move: float = 0.1
    budget: int = 1 << 30
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
    # trigger (ii): 1 = a changed voxel within trig_radius voxels (r_u = 3v),
    # among at most trig_sample changed voxels drawn per frame (0: all of
    # them); 0 = the brick rule, a superset
    trig_exact: int = 1
    trig_radius: int = 3
    trig_sample: int = 256

    def _c(self) -> _PtsConfig:
        c = _PtsConfig()
        for k, _ in _PtsConfig._fields_:
            setattr(c, k, getattr(self, k))
        return c


class PointSet:
    """The oracle's stateful point layer over one oracle Map."""

    def __init__(self, mp: "Map", pc: PointsConfig, tool: "Tool", dirs: np.ndarray):
        self._lib = _load()
        self._map = mp
        self._dirs = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
        self._pc = pc._c()
        self._tc = tool._c()
        self._h = self._lib.or_pts_new(mp._h, C.byref(self._pc), C.byref(self._tc),
                                       _ptr(self._dirs), len(self._dirs))

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_pts_free(self._h)
            self._h = None

    def frame(self, pts: np.ndarray, pose) -> int:
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, 3)
        pose = np.ascontiguousarray(pose, np.float32).reshape(16)
        return int(self._lib.or_pts_frame(self._h, self._map._h, _ptr(pts), len(pts), _ptr(pose)))

    def drain(self, max_evals: int) -> int:
        return int(self._lib.or_pts_drain(self._h, self._map._h, max_evals))

    def __len__(self):
        return int(self._lib.or_pts_count(self._h))

    def export(self) -> dict:
        n = len(self)
        out = dict(ijk=np.zeros((n, 3), np.int32), normal=np.zeros((n, 3), np.float32),
                   label=np.zeros(n, np.uint8), score=np.zeros(n, np.int16),
                   best=np.zeros(n, np.int16), a=np.zeros(n, np.float32),
                   queued=np.zeros(n, np.uint8), nviews=np.zeros(n, np.int32))
        if n:
            self._lib.or_pts_export(self._h, *(_ptr(out[k]) for k in
                                               ("ijk", "normal", "label", "score", "best", "a",
                                                "queued", "nviews")))
        return out


def octa_bin(d, bins: int) -> int:
    """Octahedral range-image cell of a sensor-frame direction."""
    lib = _load()
    d = np.ascontiguousarray(d, np.float32).reshape(3)
    return int(lib.or_octa_bin(_ptr(d), int(bins)))


def jacobi3(A: np.ndarray, sweeps: int = 8):
    """(eigenvalues, eigenvectors as columns) of a symmetric 3 x 3 matrix by
    the oracle's cyclic Jacobi routine, single precision."""
    lib = _load()
    A = np.ascontiguousarray(A, np.float32).reshape(9)
    ev = np.zeros(3, np.float32)
    V = np.zeros(9, np.float32)
    lib.or_jacobi3(_ptr(A), sweeps, _ptr(ev), _ptr(V))
    return ev, V.reshape(3, 3)


def pts_state_step(pc: PointsConfig, n_c: int, state: dict, s: int, g: int, c: float) -> dict:
    """One evaluation's state update (score, best, a, label) by the oracle."""
    lib = _load()
    cc = pc._c()
    sc = np.array([state["score"]], np.int16)
    bs = np.array([state["best"]], np.int16)
    a = np.array([state["a"]], np.float32)
    lab = np.array([state.get("label", 0)], np.uint8)
    lib.or_pts_state_step(C.byref(cc), n_c, s, g, c, _ptr(sc), _ptr(bs), _ptr(a), _ptr(lab))
    return dict(score=int(sc[0]), best=int(bs[0]), a=float(a[0]), label=int(lab[0]))


def mix64(z: int) -> int:
    """splitmix64's output function as the oracle computes it (the hash that
    draws the sample of changed voxels for the re-evaluation trigger)."""
    return int(_load().or_mix64(z & 0xFFFFFFFFFFFFFFFF))
