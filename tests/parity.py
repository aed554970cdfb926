"""Helpers shared by the GPU parity tests: the same workload parameters and
inputs handed to the CUDA path (through the C ABI) and to the oracle."""
import numpy as np

import oracle
from paper_2608_06412_gb300 import af
from paper_2608_06412_gb300.workload import Workload

FIELDS = ("ijk", "S", "w", "cleared", "occ", "known")


def oracle_config(W: Workload, **over) -> oracle.Config:
    p = dict(W.map_params())
    p.update(over)
    return oracle.Config(v=p["v"], tau=p["tau"], r_c=p["r_c"], cube_radius=p["cube_radius"],
                         clear_samples=p["clear_samples"],
                         dom_min=tuple(8 * b for b in W.dom_min),
                         dom_size=tuple(8 * b for b in W.dom_bricks),
                         cone_cos=p["cone_cos"], range_min=p["range_min"],
                         range_max=p["range_max"], clear_lo=p["clear_lo"],
                         clear_hi=p["clear_hi"], w_min=p["w_min"], w_cap=p["w_cap"],
                         clamp_signed=int(p.get("clamp_signed", 0)))


def oracle_tool(W: Workload, **over) -> oracle.Tool:
    t = W.tool()
    t.update(over)
    return oracle.Tool(**t)


def gpu_map(W: Workload, **caps) -> af.Map:
    return af.Map(W.af_config(**caps))


def gpu_voxels(m: af.Map) -> dict:
    return af.export_voxels(m.export_blocks())


def oracle_voxels(om: oracle.Map) -> dict:
    """Voxels that carry state (w > 0 or cleared), sorted by (z, y, x)."""
    e = om.export()
    keep = (e["w"] > 0) | (e["cleared"] != 0)
    return {k: v[keep] for k, v in e.items()}


def assert_maps_equal(g: dict, o: dict):
    assert len(g["ijk"]) == len(o["ijk"]), (len(g["ijk"]), len(o["ijk"]))
    np.testing.assert_array_equal(g["ijk"], o["ijk"])
    for k in FIELDS[1:]:
        bad = np.nonzero(g[k].astype(np.int64) != o[k].astype(np.int64))[0]
        assert len(bad) == 0, f"{k}: {len(bad)} voxels differ, first at {g['ijk'][bad[0]]}: " \
                              f"gpu {g[k][bad[0]]} oracle {o[k][bad[0]]}"


def to_dev(a, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def near_returns(frames, centres, radius):
    """Per frame (sensor-frame returns, pose), the returns within `radius` of
    any centre (world frame): every return that can affect what is sampled
    there, in stream order."""
    from scipy.spatial import cKDTree
    tree = cKDTree(np.asarray(centres, np.float64))
    out = []
    for fr in frames:
        d, _ = tree.query(fr.world, distance_upper_bound=radius)
        sel = np.isfinite(d)
        out.append((np.ascontiguousarray(fr.pts[sel]), np.asarray(fr.pose)))
    return out


def oracle_cluster_labels(job):
    """Oracle labels and best directions of a point cluster, from the returns
    near it (a process-pool job: config, tool, directions, scans, points and
    normals as plain values)."""
    cfg, tool, dirs, scans, pts, nrm = job
    om = oracle.Map(cfg)
    for xyz, pose in scans:
        if len(xyz):
            om.integrate(xyz, pose)
    return om.score(tool, dirs, pts, nrm)


def stream_frames(job):
    """Frames 0 .. count - 1 of a workload's stream (a process-pool job)."""
    from paper_2608_06412_gb300 import workload
    W, count = job
    return [workload.pine_frame(W, f) for f in range(count)]
