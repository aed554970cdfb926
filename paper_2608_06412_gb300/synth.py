"""Seeded synthetic inputs for the Accessibility Field hot path.

This module makes the inputs that both the CUDA path and the CPU oracle
consume: scenes of analytic primitives, a double-precision ray caster,
LiDAR ray patterns (a uniform cone and a Livox-Mid-360-like rosette), the
sensor trajectory, the voxel-deduplicated surface points with their
analytic normals, and the Fibonacci approach-direction table. It holds none
of the method's arithmetic (no TSDF, no kernels, no scoring) and imports
nothing from the rest of the package, so the oracle side may import it too.

The paper evaluates on field scans and meshes that are not available; these
generators stand in for them with the shapes, sizes and value distributions
the paper describes (Sec. 3.2: Livox Mid-360 sparsity; Sec. 4.1: Halton-
pattern scans of simple objects; Sec. 4.2: a synthetic pine).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Workload parameter sets (metres). Only numbers: nothing here computes.
# ---------------------------------------------------------------------------

#: Single synthetic frame: sphere + wall + slotted plate, 20k returns, v = 2 cm.
SINGLE_FRAME = dict(
    name="single_frame_sphere_wall_slot_20k",
    v=0.02, tau=0.06, r_c=0.01, cube_radius=3, clear_samples=8,
    w_min=3, w_cap=2000, cone_cos=0.95, range_min=0.1, range_max=40.0,
    clear_lo=1.0, clear_hi=2.25,
    tool=dict(radius=0.04, length=0.25, self_excl=0.04, corr_radius=0.05,
              corr_length=1.0, cos_theta_max=0.0, n_c=5, strict=0),
    K=32, n_returns=20000, sigma=0.01, seed=1,
)

#: Streaming Mid-360-like scans of a procedural pine: 300 frames x 20k returns.
PINE_STREAM = dict(
    name="pine_stream_mid360_300x20k",
    v=0.02, tau=0.06, r_c=0.01, cube_radius=3, clear_samples=8,
    w_min=3, w_cap=2000, cone_cos=0.95, range_min=0.1, range_max=40.0,
    clear_lo=1.0, clear_hi=2.25,
    tool=dict(radius=0.04, length=0.25, self_excl=0.04, corr_radius=0.05,
              corr_length=1.0, cos_theta_max=0.0, n_c=5, strict=0),
    K=64, n_returns=20000, sigma=0.02, seed=2, frames=300,
    orbit_radius=3.0, orbit_height=2.0, frames_per_orbit=300,
)


#: Large map: 8 pines on a noisy 40 x 40 m ground, the sensor orbiting each
#: pine in turn (375 frames per pine, 3,000 frames), v = 1 cm, K = 256.
LARGE_MAP = dict(
    name="large_map_8_pines_40m_3000x20k_v1cm",
    v=0.01, tau=0.04, r_c=0.005, cube_radius=4, clear_samples=10,
    w_min=3, w_cap=2000, cone_cos=0.95, range_min=0.1, range_max=40.0,
    clear_lo=1.0, clear_hi=2.25,
    tool=dict(radius=0.04, length=0.25, self_excl=0.04, corr_radius=0.05,
              corr_length=1.5, cos_theta_max=0.0, n_c=5, strict=0),
    K=256, n_returns=20000, sigma=0.02, seed=5, frames=3000, frames_per_pine=375,
    pines=8, ground_half=20.0, ground_tile=1.0, ground_sigma=0.02,
    orbit_radius=3.0, orbit_height=2.0,
)

# ---------------------------------------------------------------------------
# Counter-free RNG helpers
# ---------------------------------------------------------------------------

def rng(seed: int, *stream: int) -> np.random.Generator:
    """Independent seeded stream for (seed, *stream)."""
    return np.random.default_rng(np.random.SeedSequence([seed, *stream]))


def fibonacci_dirs(G: int) -> np.ndarray:
    """G unit vectors on a Fibonacci sphere: z_i = 1 - (2i+1)/G,
    phi_i = i * pi * (3 - sqrt 5). Computed in double, rounded to float32."""
    i = np.arange(G, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / G
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1).astype(np.float32)


def fibonacci_hemisphere(K: int, cos_max: float = 0.0) -> np.ndarray:
    """K unit vectors on the Fibonacci cap z > cos_max around +z:
    z_i = 1 - (i + 1/2)(1 - cos_max)/K, phi_i = i * pi * (3 - sqrt 5).
    Computed in double, rounded to float32."""
    i = np.arange(K, dtype=np.float64)
    z = 1.0 - (i + 0.5) * (1.0 - cos_max) / K
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1).astype(np.float32)


def yaw_ring(D: int = 180, pitch: float = 0.0) -> np.ndarray:
    """The paper's approach set (Sec. 3.4): D yaw angles psi_d = 2 pi d / D
    at a fixed pitch (0: horizontal), u_d = (cos p cos psi, cos p sin psi,
    sin p), in yaw order. Computed in double, rounded to float32."""
    psi = 2.0 * math.pi * np.arange(D, dtype=np.float64) / D
    cp, sp = math.cos(pitch), math.sin(pitch)
    return np.stack([cp * np.cos(psi), cp * np.sin(psi), np.full(D, sp)],
                    axis=1).astype(np.float32)


# cos 70 degrees: the normal cone of the paper's approach set (Sec. 3.4)
COS_70 = float(np.float32(math.cos(math.radians(70.0))))


def halton(index: np.ndarray, base: int) -> np.ndarray:
    """Radical inverse of integer `index` in `base` (van der Corput)."""
    index = np.asarray(index, dtype=np.int64).copy()
    out = np.zeros(index.shape, np.float64)
    f = 1.0 / base
    while np.any(index > 0):
        out += f * (index % base)
        index //= base
        f /= base
    return out


_HALTON_CACHE: dict = {}


def _halton_block(start: int, m: int):
    """Halton(2,3) points start .. start+m-1 (memoised: every frame draws the
    same unrotated sequence and differs only in its rotation)."""
    key = (start, m)
    if key not in _HALTON_CACHE:
        idx = np.arange(start, start + m)
        _HALTON_CACHE[key] = (halton(idx, 2), halton(idx, 3))
    return _HALTON_CACHE[key]


# ---------------------------------------------------------------------------
# Scenes of analytic primitives and a double-precision ray caster
# ---------------------------------------------------------------------------

@dataclass
class Group:
    """Primitives with a bounding capsule (segment a-b, radius) for culling."""
    a: np.ndarray
    b: np.ndarray
    radius: float
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))   # cx cy cz r
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))     # min xyz, max xyz
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 7)))  # a xyz, b xyz, r


@dataclass
class Scene:
    groups: list
    lo: np.ndarray   # axis-aligned bounds of all geometry
    hi: np.ndarray
    clusters: list = None   # optional contiguous group ranges (start, end) culled together


_HERE = os.path.dirname(os.path.abspath(__file__))
_RC_SRC = os.path.join(_HERE, "synth_raycast.c")
_RC_LIB = os.path.join(_HERE, "libsynth_raycast.so")
_rc = None


def build_raycaster(force: bool = False) -> str:
    """Compile the C ray caster used by the scan generators."""
    if (not force and os.path.exists(_RC_LIB)
            and os.path.getmtime(_RC_LIB) >= os.path.getmtime(_RC_SRC)):
        return _RC_LIB
    tmp = _RC_LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _RC_SRC, "-lm"],
                   check=True)
    os.replace(tmp, _RC_LIB)
    return _RC_LIB


def _raycaster():
    global _rc
    if _rc is None:
        lib = ctypes.CDLL(build_raycaster())
        lib.sr_raycast.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 10 + \
            [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _rc = lib
    return _rc


def _seg_dist(p, a, b):
    ab = b - a
    ee = float(ab @ ab)
    s = 0.0 if ee < 1e-18 else min(1.0, max(0.0, float((p - a) @ ab) / ee))
    return float(np.linalg.norm(p - (a + s * ab)))


def _cluster_capsule(groups):
    """A vertical capsule through the groups' endpoints that encloses every
    group capsule (distance to a segment is convex, so the farthest point of
    a group capsule lies at an endpoint, plus its radius)."""
    ends = np.array([e for g in groups for e in (g.a, g.b)], np.float64)
    c = ends[:, :2].mean(0)
    a = np.array([c[0], c[1], ends[:, 2].min()])
    b = np.array([c[0], c[1], ends[:, 2].max()])
    r = max(max(_seg_dist(g.a, a, b), _seg_dist(g.b, a, b)) + g.radius for g in groups)
    return [*a, *b, r * (1 + 1e-9) + 1e-9]


def _packed(scene: "Scene"):
    if getattr(scene, "_packed", None) is None:
        gs = scene.groups
        caps = np.array([[*g.a, *g.b, g.radius] for g in gs], np.float64).reshape(-1, 7)
        if scene.clusters:
            ranges = list(scene.clusters)
            assert ranges[0][0] == 0 and ranges[-1][1] == len(gs)
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(len(ranges) - 1))
            cl_caps = np.array([_cluster_capsule(gs[a:b]) for a, b in ranges], np.float64)
            cl_off = np.array([r[0] for r in ranges] + [len(gs)], np.int64)
        else:
            cl_caps = np.array([[0, 0, 0, 0, 0, 0, np.inf]], np.float64)
            cl_off = np.array([0, len(gs)], np.int64)
        out = [np.ascontiguousarray(cl_caps), cl_off, np.ascontiguousarray(caps)]
        for attr, width in (("spheres", 4), ("boxes", 6), ("cylinders", 7)):
            arrs = [np.asarray(getattr(g, attr), np.float64).reshape(-1, width) for g in gs]
            off = np.zeros(len(gs) + 1, np.int64)
            off[1:] = np.cumsum([len(a) for a in arrs])
            cat = np.concatenate(arrs) if off[-1] else np.zeros((1, width))
            out += [off, np.ascontiguousarray(cat, np.float64)]
        object.__setattr__(scene, "_packed", out)
    return getattr(scene, "_packed")


def raycast(scene: "Scene", o: np.ndarray, d: np.ndarray):
    """First hit of rays o + t d (d unit). Returns (t, unit outward normal),
    t = inf where nothing is hit. Double precision throughout."""
    o = np.ascontiguousarray(o, np.float64).reshape(3)
    d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
    n = len(d)
    t = np.full(n, np.inf)
    nrm = np.zeros((n, 3))
    if n == 0 or not scene.groups:
        return t, nrm
    clc, clo, caps, so, sp, bo, bx, co, cy = _packed(scene)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _raycaster().sr_raycast(len(clc), p(clc), p(clo), p(caps), p(so), p(sp), p(bo), p(bx),
                            p(co), p(cy), p(o), n, p(d), p(t), p(nrm))
    return t, nrm


def _bounds(groups):
    lo = np.min([np.minimum(g.a, g.b) - g.radius for g in groups], axis=0)
    hi = np.max([np.maximum(g.a, g.b) + g.radius for g in groups], axis=0)
    return lo, hi


def sphere_wall_slot_scene() -> Scene:
    """Sphere r = 0.3 m at (2,0,0); a 1x1 m wall at x = 2.6 facing -x; a
    0.4x0.4 m plate (4 cm thick) at x = 1.5 with a vertical 3 cm slot through
    its centre."""
    sph = Group(a=np.array([2.0, 0, 0]), b=np.array([2.0, 0, 0]), radius=0.31,
                spheres=np.array([[2.0, 0.0, 0.0, 0.3]]))
    wall = Group(a=np.array([2.61, 0, -0.5]), b=np.array([2.61, 0, 0.5]), radius=0.75,
                 boxes=np.array([[2.6, -0.5, -0.5, 2.62, 0.5, 0.5]]))
    plate = Group(a=np.array([1.52, 0, -0.2]), b=np.array([1.52, 0, 0.2]), radius=0.3,
                  boxes=np.array([[1.5, -0.2, -0.2, 1.54, -0.015, 0.2],
                                  [1.5, 0.015, -0.2, 1.54, 0.2, 0.2]]))
    groups = [sph, wall, plate]
    lo, hi = _bounds(groups)
    return Scene(groups, lo, hi)


def pine_scene(seed: int) -> Scene:
    """Procedural pine: trunk r = 0.2 m, h = 12 m; 6 whorls evenly spaced over
    3-11 m of 5 branches (azimuth 72 deg + U(+-10 deg), radius U(1,4) cm,
    length U(1,3) m, pitch U(30,60) deg); needle clusters every 0.3 m along
    each branch, 40 spheres of r = 5 mm ~ N(centre, 5 cm)."""
    g = rng(seed, 11)
    groups = [Group(a=np.array([0.0, 0, 0]), b=np.array([0.0, 0, 12.0]), radius=0.2,
                    cylinders=np.array([[0, 0, 0, 0, 0, 12.0, 0.2]]))]
    for wi, z in enumerate(np.linspace(3.0, 11.0, 6)):
        rot = g.uniform(0, 2 * math.pi)
        for bi in range(5):
            az = rot + math.radians(72.0 * bi + g.uniform(-10, 10))
            rb = g.uniform(0.01, 0.04)
            ln = g.uniform(1.0, 3.0)
            pitch = math.radians(g.uniform(30, 60))
            dvec = np.array([math.cos(pitch) * math.cos(az), math.cos(pitch) * math.sin(az),
                             math.sin(pitch)])
            a = np.array([0.0, 0.0, z])
            b = a + ln * dvec
            centres = [a + s * dvec for s in np.arange(0.3, ln + 1e-9, 0.3)]
            needles = []
            for c in centres:
                off = g.normal(0.0, 0.05, size=(40, 3))
                needles.append(np.concatenate([c[None] + off, np.full((40, 1), 0.005)], 1))
            spheres = np.concatenate(needles, 0) if needles else np.zeros((0, 4))
            reach = 0.0
            if len(spheres):
                rel = spheres[:, :3] - a
                s = np.clip(rel @ dvec / ln, 0.0, 1.0)
                dist = np.linalg.norm(rel - (s[:, None] * ln) * dvec[None], axis=1)
                reach = float(dist.max()) + 0.005
            groups.append(Group(a=a, b=b, radius=max(rb, reach) + 1e-3,
                                spheres=spheres,
                                cylinders=np.array([[*a, *b, rb]])))
    lo, hi = _bounds(groups)
    return Scene(groups, lo, hi)


# ---------------------------------------------------------------------------
# Frames: returns in the sensor frame, the pose, and the scored point set
# ---------------------------------------------------------------------------

@dataclass
class Frame:
    pts: np.ndarray       # (n,3) float32 returns, sensor frame
    pose: np.ndarray      # (4,4) float32 world_from_sensor, row-major
    world: np.ndarray     # (n,3) float64 returns, world frame
    normal: np.ndarray    # (n,3) float64 analytic outward normal at each hit


def pine_positions(seed: int, count: int, half: float):
    """Pine positions: a jittered 4 x 2 grid over the square of half-width
    `half` (x in 4 columns, y in 2 rows), jitter U(+-1 m)."""
    g = rng(seed, 71)
    cols, rows = 4, max(1, (count + 3) // 4)
    out = []
    for k in range(count):
        cx = -half + (2 * half) * ((k % cols) + 0.5) / cols
        cy = -half + (2 * half) * ((k // cols) + 0.5) / rows
        out.append((cx + g.uniform(-1, 1), cy + g.uniform(-1, 1)))
    return np.array(out)


def forest_ground_scene(seed: int, count: int = 8, half: float = 20.0, tile: float = 1.0,
                        ground_sigma: float = 0.02) -> Scene:
    """`count` procedural pines (pine_scene(seed * 100 + k)) at
    pine_positions, on a ground of square tiles of edge `tile` covering
    [-half, half]^2, each tile's top at height N(0, ground_sigma); one group
    per tile row."""
    groups, clusters = [], []
    for k, (cx, cy) in enumerate(pine_positions(seed, count, half)):
        start = len(groups)
        off = np.array([cx, cy, 0.0])
        for gr in pine_scene(seed * 100 + k).groups:
            sp = gr.spheres.copy()
            if len(sp):
                sp[:, :3] += off
            cy_ = gr.cylinders.copy()
            if len(cy_):
                cy_[:, :3] += off
                cy_[:, 3:6] += off
            groups.append(Group(a=gr.a + off, b=gr.b + off, radius=gr.radius, spheres=sp,
                                boxes=gr.boxes, cylinders=cy_))
        clusters.append((start, len(groups)))
    g = rng(seed, 73)
    n = int(round(2 * half / tile))
    for r in range(n):
        y0 = -half + r * tile
        tops = g.normal(0.0, ground_sigma, n)
        boxes = np.array([[-half + c * tile, y0, -0.2, -half + (c + 1) * tile, y0 + tile, tops[c]]
                          for c in range(n)])
        zc, hz = (tops.max() - 0.2) / 2, (tops.max() + 0.2) / 2
        groups.append(Group(a=np.array([-half, y0 + tile / 2, zc]),
                            b=np.array([half, y0 + tile / 2, zc]),
                            radius=math.hypot(tile / 2, hz) + 1e-3, boxes=boxes))
        clusters.append((len(groups) - 1, len(groups)))
    lo, hi = _bounds(groups)
    return Scene(groups, lo, hi, clusters)


def yaw_pose(origin, yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    T = np.eye(4)
    T[:3, :3] = [[c, -s, 0], [s, c, 0], [0, 0, 1]]
    T[:3, 3] = origin
    return T


def _finish(T: np.ndarray, world: np.ndarray, normal: np.ndarray) -> Frame:
    R, t = T[:3, :3], T[:3, 3]
    pts = ((world - t) @ R).astype(np.float32)        # R^T (p - t)
    return Frame(pts=pts, pose=T.astype(np.float32), world=world, normal=normal)


def cone_frame(scene: Scene, n_hits: int, sigma: float, seed: int,
               origin=(0.0, 0.0, 0.0)) -> Frame:
    """Rays drawn uniformly over the cone from `origin` that bounds the scene,
    until n_hits returns; range noise N(0, sigma)."""
    g = rng(seed, 21)
    o = np.asarray(origin, np.float64)
    corners = np.array([[x, y, z] for x in (scene.lo[0], scene.hi[0])
                        for y in (scene.lo[1], scene.hi[1])
                        for z in (scene.lo[2], scene.hi[2])]) - o
    axis = (scene.lo + scene.hi) / 2 - o
    axis /= np.linalg.norm(axis)
    cos_a = float(np.min(corners @ axis / np.linalg.norm(corners, axis=1)))
    helper = np.array([0.0, 0, 1]) if abs(axis[2]) < 0.9 else np.array([1.0, 0, 0])
    e1 = np.cross(axis, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(axis, e1)
    world, normal = [], []
    have = 0
    while have < n_hits:
        m = 32768
        cz = g.uniform(cos_a, 1.0, m)
        ph = g.uniform(0.0, 2 * math.pi, m)
        sz = np.sqrt(1 - cz * cz)
        d = cz[:, None] * axis + (sz * np.cos(ph))[:, None] * e1 + (sz * np.sin(ph))[:, None] * e2
        noise = g.normal(0.0, sigma, m)
        t, nr = raycast(scene, o, d)
        ok = np.isfinite(t)
        world.append(o + (t[ok] + noise[ok])[:, None] * d[ok])
        normal.append(nr[ok])
        have += int(ok.sum())
    world = np.concatenate(world)[:n_hits]
    normal = np.concatenate(normal)[:n_hits]
    return _finish(yaw_pose(o, 0.0), world, normal)


def rosette_frame(scene: Scene, frame: int, seed: int, n_hits: int = 20000,
                  sigma: float = 0.02, orbit_radius: float = 3.0,
                  orbit_height: float = 2.0, frames_per_orbit: int = 300,
                  el_lo: float = -7.0, el_hi: float = 52.0,
                  range_lo: float = 0.1, range_hi: float = 40.0,
                  centre=(0.0, 0.0)) -> Frame:
    """Livox-Mid-360-like frame: a Cranley-Patterson-rotated Halton(2,3)
    pattern over azimuth [0, 360) deg and elevation [el_lo, el_hi] deg, from
    a sensor orbiting `centre` (x, y); rays are drawn until n_hits returns
    with range in [range_lo, range_hi]; range noise N(0, sigma)."""
    g = rng(seed, 31, frame)
    phi = 2.0 * math.pi * frame / frames_per_orbit
    o = np.array([centre[0] + orbit_radius * math.cos(phi),
                  centre[1] + orbit_radius * math.sin(phi), orbit_height])
    T = yaw_pose(o, phi + math.pi)
    shift = g.uniform(0.0, 1.0, 2)
    world, normal = [], []
    have, start = 0, 1
    while have < n_hits:
        m = 65536
        h2, h3 = _halton_block(start, m)
        start += m
        az = 2 * math.pi * np.mod(h2 + shift[0], 1.0)
        el = np.radians(el_lo + (el_hi - el_lo) * np.mod(h3 + shift[1], 1.0))
        ds = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], 1)
        d = ds @ T[:3, :3].T
        t, nr = raycast(scene, o, d)
        ok = np.isfinite(t) & (t >= range_lo) & (t <= range_hi)
        noise = g.normal(0.0, sigma, m)
        world.append(o + (t[ok] + noise[ok])[:, None] * d[ok])
        normal.append(nr[ok])
        have += int(ok.sum())
    world = np.concatenate(world)[:n_hits]
    normal = np.concatenate(normal)[:n_hits]
    return _finish(T, world, normal)


def surface_points(world: np.ndarray, normal: np.ndarray, v: float):
    """Voxel-deduplicated surface points (Sec. 3.1): one point per voxel that
    holds a return, in order of first occurrence, placed at the voxel centre,
    with the analytic normal of that first return. Returns float32 arrays."""
    vv = float(np.float32(v))
    idx = np.floor(world / vv).astype(np.int64)
    _, first = np.unique(idx, axis=0, return_index=True)
    first = np.sort(first)
    pts = ((idx[first] + 0.5) * vv).astype(np.float32)
    return pts, normal[first].astype(np.float32)


def domain_bricks(lo, hi, v: float, margin: float, edge: int = 8):
    """Brick-aligned voxel box covering [lo - margin, hi + margin]:
    returns (min corner in bricks, size in bricks)."""
    b = v * edge
    bmin = np.floor((np.asarray(lo) - margin) / b).astype(int)
    bmax = np.floor((np.asarray(hi) + margin) / b).astype(int)
    return tuple(int(x) for x in bmin), tuple(int(x) for x in (bmax - bmin + 1))
