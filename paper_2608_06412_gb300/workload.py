"""Synthetic workloads as plain parameters: scene, frames, map box, tool and
direction table. Consumers turn the parameter dicts into their own config
structs (af.MapConfig for the library; the test-suite builds the oracle's).
Nothing here computes any part of the method.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import synth

MAP_KEYS = ("v", "tau", "r_c", "cube_radius", "clear_samples", "cone_cos", "range_min",
            "range_max", "clear_lo", "clear_hi", "w_min", "w_cap")


@dataclass
class Workload:
    name: str
    params: dict              # synth.SINGLE_FRAME / PINE_STREAM style dict
    scene: synth.Scene
    dom_min: tuple            # map box, bricks
    dom_bricks: tuple
    dirs: np.ndarray          # (2K, 3) float32 Fibonacci table

    def map_params(self) -> dict:
        return {k: self.params[k] for k in MAP_KEYS}

    def tool(self) -> dict:
        return dict(self.params["tool"])

    def af_config(self, **caps):
        from .af import MapConfig
        p = self.params
        kw = dict(voxel_size=p["v"], truncation=p["tau"], r_c=p["r_c"],
                  cube_radius=p["cube_radius"], clear_samples=p["clear_samples"],
                  domain_min=self.dom_min, domain_bricks=self.dom_bricks,
                  cone_cos=p["cone_cos"], range_min=p["range_min"],
                  range_max=p["range_max"], clear_lo=p["clear_lo"],
                  clear_hi=p["clear_hi"], w_min=p["w_min"], w_cap=p["w_cap"])
        kw.update(caps)     # capacities, and overrides of the above
        return MapConfig(**kw)

    def af_tool(self):
        from .af import ToolConfig
        return ToolConfig(**self.tool())


def single_frame(seed: int | None = None) -> Workload:
    """Sphere + wall + slotted plate, one frame of 20k returns (v = 2 cm)."""
    p = dict(synth.SINGLE_FRAME)
    if seed is not None:
        p["seed"] = seed
    sc = synth.sphere_wall_slot_scene()
    lo = np.minimum(sc.lo, 0.0)
    hi = np.maximum(sc.hi, 0.0)
    dmin, db = synth.domain_bricks(lo, hi, p["v"], margin=0.5)
    return Workload(p["name"], p, sc, dmin, db, synth.fibonacci_dirs(2 * p["K"]))


def single_frame_inputs(W: Workload, n: int | None = None):
    """(frame, surface points, normals) of the single-frame workload."""
    p = W.params
    fr = synth.cone_frame(W.scene, n or p["n_returns"], p["sigma"], p["seed"])
    pts, nrm = synth.surface_points(fr.world, fr.normal, p["v"])
    return fr, pts, nrm


def pine_stream(seed: int | None = None) -> Workload:
    """Procedural pine orbited by a Mid-360-like sensor, 20k returns / frame."""
    p = dict(synth.PINE_STREAM)
    if seed is not None:
        p["seed"] = seed
    sc = synth.pine_scene(p["seed"])
    r = p["orbit_radius"] + 0.5
    lo = np.minimum(sc.lo, [-r, -r, 0.0])
    hi = np.maximum(sc.hi, [r, r, p["orbit_height"]])
    dmin, db = synth.domain_bricks(lo, hi, p["v"], margin=0.5)
    return Workload(p["name"], p, sc, dmin, db, synth.fibonacci_dirs(2 * p["K"]))


def pine_frame(W: Workload, f: int):
    """Frame f of the pine stream: (frame, surface points, normals)."""
    p = W.params
    fr = synth.rosette_frame(W.scene, f, p["seed"], n_hits=p["n_returns"], sigma=p["sigma"],
                             orbit_radius=p["orbit_radius"], orbit_height=p["orbit_height"],
                             frames_per_orbit=p["frames_per_orbit"])
    pts, nrm = synth.surface_points(fr.world, fr.normal, p["v"])
    return fr, pts, nrm


def large_map(seed: int | None = None) -> Workload:
    """8 pines on a noisy 40 x 40 m ground, 3,000 frames (375 orbit frames
    around each pine), v = 1 cm, tau = 4 cm, K = 256, corridor 1.5 m."""
    p = dict(synth.LARGE_MAP)
    if seed is not None:
        p["seed"] = seed
    sc = synth.forest_ground_scene(p["seed"], p["pines"], p["ground_half"], p["ground_tile"],
                                   p["ground_sigma"])
    lo = np.minimum(sc.lo, [-p["ground_half"], -p["ground_half"], -0.3])
    hi = np.maximum(sc.hi, [p["ground_half"], p["ground_half"], p["orbit_height"]])
    dmin, db = synth.domain_bricks(lo, hi, p["v"], margin=0.1)
    return Workload(p["name"], p, sc, dmin, db, synth.fibonacci_dirs(2 * p["K"]))


def large_frame(W: Workload, f: int):
    """Frame f of the large map: the sensor orbits pine f // frames_per_pine.
    Returns (frame, surface points, normals)."""
    p = W.params
    centre = synth.pine_positions(p["seed"], p["pines"], p["ground_half"])[f // p["frames_per_pine"]]
    fr = synth.rosette_frame(W.scene, f, p["seed"], n_hits=p["n_returns"], sigma=p["sigma"],
                             orbit_radius=p["orbit_radius"], orbit_height=p["orbit_height"],
                             frames_per_orbit=p["frames_per_pine"], centre=centre)
    pts, nrm = synth.surface_points(fr.world, fr.normal, p["v"])
    return fr, pts, nrm


def _large_frames_chunk(args):
    seed, fs = args
    W = large_map(seed)
    out = []
    for f in fs:
        fr, pts, nrm = large_frame(W, f)
        out.append((fr.pts, fr.pose, fr.world.astype(np.float32), pts, nrm))
    return out


def large_frames(W: Workload, frames, workers: int = 0):
    """Frames of the large map as (sensor-frame returns, pose, world returns
    (float32), surface points, normals), generated by `workers` spawned
    processes (0: os.cpu_count()). Start it before any CUDA call."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import os
    frames = list(frames)
    workers = workers or os.cpu_count() or 1
    chunks = [frames[i::workers] for i in range(workers)]
    env = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_large_frames_chunk, [(W.params["seed"], c) for c in chunks]))
    finally:
        if env is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env
    by = {}
    for c, part in zip(chunks, parts):
        for f, item in zip(c, part):
            by[f] = item
    return [by[f] for f in frames]


def soft_points(frames, v: float, count: int = 100_000, seed: int = 0):
    """Surface points of the differentiable-form workload: one point (and
    normal) per voxel that the stream's surface points fall in, its first
    occurrence in stream order, then `count` of them drawn without
    replacement by a seeded generator (all of them if fewer)."""
    pts = np.concatenate([f[1] for f in frames])
    nrm = np.concatenate([f[2] for f in frames])
    ijk = np.floor(pts.astype(np.float64) / np.float64(np.float32(v))).astype(np.int64)
    _, first = np.unique(ijk, axis=0, return_index=True)
    first = np.sort(first)
    g = synth.rng(seed, 61)
    pick = np.sort(g.choice(len(first), min(count, len(first)), replace=False))
    sel = first[pick]
    return np.ascontiguousarray(pts[sel]), np.ascontiguousarray(nrm[sel])

#: Map capacities the benchmark uses for the pine stream (and the full-size
#: parity test runs with): 512k hash slots, 256k bricks (1.1 GB), 64k returns
#: and points per call.
BENCH_CAPS = dict(hash_capacity=1 << 19, pool_blocks=1 << 18, max_returns=1 << 16,
                  max_points=1 << 16)


#: The three tools of the batched workload: cylinder radius r and length L,
#: corridor length; the corridor radius is r + 1 cm and r_s = r, as for the
#: 4 cm tool of the single-scene workloads.
BATCH_TOOLS = [dict(radius=0.03, length=0.15, self_excl=0.03, corr_radius=0.04,
                    corr_length=0.5, cos_theta_max=0.0, n_c=5, strict=0),
               dict(radius=0.04, length=0.25, self_excl=0.04, corr_radius=0.05,
                    corr_length=1.0, cos_theta_max=0.0, n_c=5, strict=0),
               dict(radius=0.06, length=0.40, self_excl=0.06, corr_radius=0.07,
                    corr_length=1.5, cos_theta_max=0.0, n_c=5, strict=0)]


def clutter_scene(seed: int) -> synth.Scene:
    """Boxes (5-40 cm) and spheres (r 5-25 cm) scattered over 3 x 3 x 2 m."""
    g = synth.rng(seed, 41)
    groups = []
    for _ in range(20):
        c = g.uniform([-1.5, -1.5, 0.0], [1.5, 1.5, 2.0])
        h = g.uniform(0.025, 0.2, 3)
        groups.append(synth.Group(a=c, b=c, radius=float(np.linalg.norm(h)) + 1e-3,
                                  boxes=np.array([[*(c - h), *(c + h)]])))
    for _ in range(20):
        c = g.uniform([-1.5, -1.5, 0.0], [1.5, 1.5, 2.0])
        r = float(g.uniform(0.05, 0.25))
        groups.append(synth.Group(a=c, b=c, radius=r + 1e-3, spheres=np.array([[*c, r]])))
    lo, hi = synth._bounds(groups)
    return synth.Scene(groups, lo, hi)


def forest_scene(seed: int, count: int) -> synth.Scene:
    """`count` procedural pines within 2.5 m of the origin."""
    g = synth.rng(seed, 43)
    groups = []
    for k in range(count):
        off = np.zeros(3) if k == 0 else np.r_[g.uniform(-2.5, 2.5, 2), 0.0]
        for gr in synth.pine_scene(seed * 100 + k).groups:
            sp = gr.spheres.copy()
            if len(sp):
                sp[:, :3] += off
            cy = gr.cylinders.copy()
            if len(cy):
                cy[:, :3] += off
                cy[:, 3:6] += off
            groups.append(synth.Group(a=gr.a + off, b=gr.b + off, radius=gr.radius,
                                      spheres=sp, boxes=gr.boxes, cylinders=cy))
    lo, hi = synth._bounds(groups)
    return synth.Scene(groups, lo, hi)


def batch_scenes(count: int = 64, seed: int = 3, n_lo: int = 2000, n_hi: int = 60000):
    """Scenes of the batched workload: 1-4 pines or box/sphere clutter,
    returns per frame ~ U[n_lo, n_hi], one of three tools, K in {16, 64, 128};
    each scene orbited by its own Mid-360-like sensor."""
    g = synth.rng(seed, 51)
    out = []
    for s in range(count):
        p = dict(synth.PINE_STREAM)
        kind = int(g.integers(0, 5))           # 0 clutter, 1-4 pines
        sc = clutter_scene(seed * 1000 + s) if kind == 0 else forest_scene(seed * 1000 + s, kind)
        p["tool"] = dict(BATCH_TOOLS[int(g.integers(0, 3))])
        p["K"] = int(g.choice([16, 64, 128]))
        p["n_returns"] = int(g.integers(n_lo, n_hi + 1))
        p["seed"] = seed * 1000 + s
        p["orbit_radius"] = 3.0 if kind <= 1 else 5.5
        p["name"] = f"batch_scene_{s}"
        r = p["orbit_radius"] + 0.5
        lo = np.minimum(sc.lo, [-r, -r, 0.0])
        hi = np.maximum(sc.hi, [r, r, p["orbit_height"]])
        dmin, db = synth.domain_bricks(lo, hi, p["v"], margin=0.5)
        out.append(Workload(p["name"], p, sc, dmin, db, synth.fibonacci_dirs(2 * p["K"])))
    return out
