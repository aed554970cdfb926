"""Batched ticks (af_batch_*): scenes of uneven size, with their own tools and
direction tables, ticked together must give exactly what the per-scene path
(af_integrate_scan + af_score) gives -- labels, best directions and maps --
under every launch shape the autotuner tries."""
import numpy as np
import pytest

from parity import gpu_voxels, to_dev
from paper_2608_06412_gb300 import af, workload

pytestmark = pytest.mark.gpu

CAPS = dict(hash_capacity=1 << 17, pool_blocks=1 << 15, max_returns=1 << 14,
            max_points=1 << 14)


@pytest.fixture(scope="module")
def scenes():
    S = workload.batch_scenes(6, seed=9, n_lo=300, n_hi=4000)
    return S


def _items(S, f, empty=2, no_points=4):
    """Frame f of every scene; scene `empty` has no returns and no points,
    scene `no_points` integrates but scores nothing."""
    import torch
    out = []
    for s, W in enumerate(S):
        fr, pts, nrm = workload.pine_frame(W, f)
        xyz = fr.pts if s != empty else fr.pts[:0]
        if s in (empty, no_points):
            pts, nrm = pts[:0], nrm[:0]
        out.append((to_dev(xyz), fr.pose, to_dev(pts), to_dev(nrm),
                    torch.empty(len(pts), dtype=torch.uint8, device="cuda"),
                    torch.empty(len(pts), dtype=torch.int16, device="cuda")))
    return out


def test_batch_ticks_equal_per_scene_path(scenes):
    """Odd scenes use the [-tau, tau] clamp, so one batch mixes both clamps."""
    import torch
    S = scenes
    plain = [af.Map(W.af_config(clamp_signed=s % 2, **CAPS)) for s, W in enumerate(S)]
    mapsb = [af.Map(W.af_config(clamp_signed=s % 2, **CAPS)) for s, W in enumerate(S)]
    for W, a, b in zip(S, plain, mapsb):
        a.set_tool(W.af_tool(), W.dirs)
        b.set_tool(W.af_tool(), W.dirs)
    batch = af.Batch(mapsb)
    ticks = 22                       # 9 shapes x 2 timed ticks, then the chosen one
    for f in range(ticks):
        items = _items(S, f)
        batch.tick(items)
        ref = []
        for (xyz, pose, pts, nrm, _, _), mp in zip(items, plain):
            mp.integrate_scan(xyz, pose)
            ref.append(mp.score(pts, nrm) if len(pts) else None)
        torch.cuda.synchronize()
        for s, (it, r) in enumerate(zip(items, ref)):
            if r is None:
                continue
            np.testing.assert_array_equal(it[4].cpu().numpy(), r[0].cpu().numpy(), f"tick {f} scene {s}")
            np.testing.assert_array_equal(it[5].cpu().numpy(), r[1].cpu().numpy(), f"tick {f} scene {s}")
    for s, (a, b) in enumerate(zip(plain, mapsb)):
        va, vb = gpu_voxels(a), gpu_voxels(b)
        for k in va:
            np.testing.assert_array_equal(va[k], vb[k], f"scene {s} field {k}")
        assert ((va["S"] < 0).any() == bool(s % 2)) or len(va["S"]) == 0
        assert a.stats()["tests"] == b.stats()["tests"]
        assert a.stats()["returns_accepted"] == b.stats()["returns_accepted"]
    t = batch.tuning()
    assert t["explored"] == 9 and t["done"]
    assert t["returns_per_tile"] in (8, 16, 32) and t["warps_per_cta"] in (2, 4, 8)
    # the labels actually exercise both outcomes
    allab = np.concatenate([it[4].cpu().numpy() for it in items])
    assert (allab == af.ACCESSIBLE).any() and (allab == af.BLOCKED).any()


def test_batch_fixed_shape_and_argument_errors(scenes):
    import torch
    S = scenes[:3]
    maps = [af.Map(W.af_config(**CAPS)) for W in S]
    for W, m in zip(S, maps):
        m.set_tool(W.af_tool(), W.dirs)
    batch = af.Batch(maps)
    batch.set_tuning(32, 8)
    batch.tick(_items(S, 0, empty=-1, no_points=-1))
    torch.cuda.synchronize()
    t = batch.tuning()
    assert (t["returns_per_tile"], t["warps_per_cta"], t["done"]) == (32, 8, True)
    with pytest.raises(af.AfError):
        batch.set_tuning(12, 8)
    with pytest.raises(af.AfError):
        af.Batch([maps[0], maps[0]])
    other = af.Map(S[0].af_config(**CAPS))      # no tool: scoring must be refused
    b2 = af.Batch([other])
    with pytest.raises(af.AfError) as e:
        b2.tick(_items(S[:1], 0, empty=-1, no_points=-1))
    assert e.value.status == af.ERR_STATE


def test_batch_many_tiny_scenes_share_warps():
    """40 scenes of 2-12 returns: nearly every allocation warp holds lanes of
    several maps, so per-map bookkeeping (dirty lists, counters) must not
    mix maps. Maps and labels equal the per-scene path's after every tick."""
    import torch
    S = workload.batch_scenes(40, seed=17, n_lo=2, n_hi=12)
    caps = dict(hash_capacity=1 << 12, pool_blocks=1 << 10, max_returns=64, max_points=64)
    plain = [af.Map(W.af_config(**caps)) for W in S]
    mapsb = [af.Map(W.af_config(**caps)) for W in S]
    for W, a, b in zip(S, plain, mapsb):
        a.set_tool(W.af_tool(), W.dirs)
        b.set_tool(W.af_tool(), W.dirs)
    batch = af.Batch(mapsb)
    batch.set_tuning(8, 2)
    rng = np.random.default_rng(3)
    for f in range(6):
        items = []
        for W in S:
            fr, pts, nrm = workload.pine_frame(W, f)
            take = rng.choice(len(fr.pts), min(len(fr.pts), W.params["n_returns"]), replace=False)
            pts, nrm = pts[:8], nrm[:8]
            items.append((to_dev(fr.pts[take]), fr.pose, to_dev(pts), to_dev(nrm),
                          torch.empty(len(pts), dtype=torch.uint8, device="cuda"),
                          torch.empty(len(pts), dtype=torch.int16, device="cuda")))
        batch.tick(items)
        ref = []
        for (xyz, pose, pts, nrm, _, _), mp in zip(items, plain):
            mp.integrate_scan(xyz, pose)
            ref.append(mp.score(pts, nrm))
        torch.cuda.synchronize()
        for s, (it, r) in enumerate(zip(items, ref)):
            np.testing.assert_array_equal(it[4].cpu().numpy(), r[0].cpu().numpy(), f"tick {f} scene {s}")
            np.testing.assert_array_equal(it[5].cpu().numpy(), r[1].cpu().numpy(), f"tick {f} scene {s}")
        for s, (a, b) in enumerate(zip(plain, mapsb)):
            va, vb = gpu_voxels(a), gpu_voxels(b)
            for k in va:
                np.testing.assert_array_equal(va[k], vb[k], f"tick {f} scene {s} field {k}")
