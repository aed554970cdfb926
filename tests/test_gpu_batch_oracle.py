"""The batched form at its workload's full size against the oracle: 64 scenes
of 1-4 pines or box / sphere clutter, 2,000-60,000 returns per frame, three
tools (r 3/4/6 cm, L 15/25/40 cm, corridors 0.5/1.0/1.5 m) and K in
{16, 64, 128}, ticked together three times (af_batch_tick, the bench's
capacities). Then, for every scene, bit for bit against the oracle:
 * S, w, cleared, occupied and known of sampled voxels;
 * labels and best directions of a cluster of the last frame's points.
The oracle builds each sample from the returns that can affect it: a voxel's
state depends only on returns whose cube holds it or whose cleared band
reaches it (within 0.25 m); a point's label only on voxels within its
kernels' reach, so on returns within L + L_c + r + 0.3 m."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from parity import (near_returns, oracle_cluster_labels, oracle_config, oracle_tool,
                    stream_frames, to_dev)
from paper_2608_06412_gb300 import af, workload

pytestmark = pytest.mark.gpu

FRAMES = 3
VOXEL_RADIUS = 0.25
CAPS = dict(hash_capacity=1 << 18, pool_blocks=1 << 16, max_returns=1 << 16, max_points=1 << 16)


def _reach(W):
    t = W.tool()
    return t["length"] + t["corr_length"] + max(t["radius"], t["corr_radius"]) + 0.3


def _pool():
    # one process per core, started with spawn: the parent holds a CUDA context
    return mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def ticked():
    import torch
    S = workload.batch_scenes(64)
    with _pool() as pool:
        frames = pool.map(stream_frames, [(W, FRAMES) for W in S])
    maps = [af.Map(W.af_config(**CAPS)) for W in S]
    for W, m in zip(S, maps):
        m.set_tool(W.af_tool(), W.dirs)
    batch = af.Batch(maps)
    for f in range(FRAMES):
        items = []
        for fs in frames:
            fr, p, n = fs[f]
            items.append((to_dev(fr.pts), fr.pose, to_dev(p), to_dev(n),
                          torch.empty(len(p), dtype=torch.uint8, device="cuda"),
                          torch.empty(len(p), dtype=torch.int16, device="cuda")))
        batch.tick(items)
    torch.cuda.synchronize()
    last = [(it[4].cpu().numpy(), it[5].cpu().numpy()) for it in items]
    assert all(m.sync_status() == 0 for m in maps)
    return S, frames, maps, last


def test_workload_is_the_batched_mix(ticked):
    S, frames, _, _ = ticked
    n = [len(fs[0][0].pts) for fs in frames]
    assert len(S) == 64 and min(n) >= 2000 and max(n) <= 60000 and max(n) > 40000
    assert {W.params["K"] for W in S} == {16, 64, 128}
    assert len({W.tool()["radius"] for W in S}) == 3


def test_batched_maps_bit_exact_on_sampled_voxels(ticked):
    S, frames, maps, _ = ticked
    rng = np.random.default_rng(11)
    checked = 0
    for W, fs, g in zip(S, frames, maps):
        gv = af.export_voxels(g.export_blocks(cap=1500))   # bricks of the first frames
        sel = rng.choice(len(gv["ijk"]), 4, replace=False)
        v = np.float64(np.float32(W.params["v"]))
        scans = near_returns([fr for fr, _, _ in fs], (gv["ijk"][sel] + 0.5) * v, VOXEL_RADIUS)
        om = oracle.Map(oracle_config(W))
        for xyz, pose in scans:
            if len(xyz):
                om.integrate(xyz, pose)
        for k in sel:
            i, j, l = (int(x) for x in gv["ijk"][k])
            S_, w, cl = om.voxel(i, j, l)
            assert (int(gv["S"][k]), int(gv["w"][k]), int(gv["cleared"][k])) == (S_, w, cl), \
                (W.name, i, j, l)
            assert int(gv["occ"][k]) == om.occ(i, j, l) and int(gv["known"][k]) == om.known(i, j, l)
            checked += 1
    assert checked == 4 * len(S)


def test_batched_labels_bit_exact_on_sampled_points(ticked):
    S, frames, _, last = ticked
    rng = np.random.default_rng(12)
    jobs, picks = [], []
    for W, fs, (lab, best) in zip(S, frames, last):
        _, pts, nrm = fs[-1]
        scored = np.nonzero(lab != af.UNSCORED)[0]
        seed = rng.choice(scored)
        near = np.argsort(np.linalg.norm(pts - pts[seed], axis=1))[:8]
        scans = near_returns([fr for fr, _, _ in fs], pts[near].astype(np.float64), _reach(W))
        jobs.append((oracle_config(W), oracle_tool(W), W.dirs, scans, pts[near], nrm[near]))
        picks.append(near)
    # the oracle's kernel tables take seconds per scene
    with _pool() as pool:
        res = pool.map(oracle_cluster_labels, jobs)
    seen = set()
    for W, near, (lab, best), (ol, ob) in zip(S, picks, last, res):
        np.testing.assert_array_equal(lab[near], ol, err_msg=W.name)
        np.testing.assert_array_equal(best[near], ob, err_msg=W.name)
        seen |= set(ol.tolist())
    assert {af.ACCESSIBLE, af.BLOCKED} <= seen
