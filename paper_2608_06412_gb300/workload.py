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
        return MapConfig(voxel_size=p["v"], truncation=p["tau"], r_c=p["r_c"],
                         cube_radius=p["cube_radius"], clear_samples=p["clear_samples"],
                         domain_min=self.dom_min, domain_bricks=self.dom_bricks,
                         cone_cos=p["cone_cos"], range_min=p["range_min"],
                         range_max=p["range_max"], clear_lo=p["clear_lo"],
                         clear_hi=p["clear_hi"], w_min=p["w_min"], w_cap=p["w_cap"], **caps)

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


#: Map capacities the benchmark uses for the pine stream (and the full-size
#: parity test runs with): 512k hash slots, 256k bricks (1.1 GB), 64k returns
#: and points per call.
BENCH_CAPS = dict(hash_capacity=1 << 19, pool_blocks=1 << 18, max_returns=1 << 16,
                  max_points=1 << 16)
