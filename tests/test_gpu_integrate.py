"""GPU parity of scan-centric TSDF integration (Sec. 3.2, 3.4, 3.6) against
the oracle: every voxel's integer weight w, fixed-point SDF sum S, cleared
bit and occupied / known bits must be identical. Also: edge cases (empty,
ragged, invalid returns, duplicates past the weight cap, the map box edge),
determinism, and the capacity error path."""
import numpy as np
import pytest

import oracle
from parity import (assert_maps_equal, gpu_map, gpu_voxels, oracle_config, oracle_voxels,
                    to_dev)
from paper_2608_06412_gb300 import af, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def single():
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    return W, fr


def _both(W, scans, **caps):
    """Integrate the same scans on the GPU and in the oracle."""
    import torch
    g = gpu_map(W, **caps)
    o = oracle.Map(oracle_config(W))
    for xyz, pose in scans:
        g.integrate_scan(to_dev(xyz.astype(np.float32)), pose)
        o.integrate(xyz, pose)
    torch.cuda.synchronize()
    return g, o


def test_single_frame_bit_exact(single):
    W, fr = single
    g, o = _both(W, [(fr.pts, fr.pose)])
    assert g.sync_status() == 0
    gv, ov = gpu_voxels(g), oracle_voxels(o)
    assert len(ov["ijk"]) > 20000
    assert_maps_equal(gv, ov)
    st = g.stats()
    assert st["returns_accepted"] == len(fr.pts)


def test_stream_with_poses_bit_exact():
    """Twelve Mid-360-like frames from an orbiting sensor (non-identity poses,
    growing map, repeated observations)."""
    W = workload.pine_stream()
    scans = []
    for f in range(0, 120, 10):
        fr, _, _ = workload.pine_frame(W, f)
        scans.append((fr.pts, fr.pose))
    g, o = _both(W, scans, hash_capacity=1 << 18, pool_blocks=1 << 17)
    assert_maps_equal(gpu_voxels(g), oracle_voxels(o))


@pytest.mark.parametrize("n", [0, 1, 31, 33, 1031])
def test_ragged_sizes(single, n):
    W, fr = single
    g, o = _both(W, [(fr.pts[:n], fr.pose)])
    assert_maps_equal(gpu_voxels(g), oracle_voxels(o))


def test_invalid_returns_and_duplicates(single):
    """NaN / inf / out-of-range returns are dropped; 2100 copies of one return
    exceed the weight cap of 2000 and are rescaled proportionally."""
    W, fr = single
    pts = fr.pts[:500].copy()
    pts[::7] = np.nan
    pts[3::11] = np.array([np.inf, 0, 0], np.float32)
    pts[5::13] = np.array([0.05, 0, 0], np.float32)       # closer than 0.1 m
    pts[6::17] = np.array([45.0, 0, 0], np.float32)       # beyond 40 m
    dup = np.repeat(fr.pts[600:601], 2100, 0)
    g, o = _both(W, [(pts, fr.pose), (dup, fr.pose), (pts[::-1].copy(), fr.pose)])
    gv, ov = gpu_voxels(g), oracle_voxels(o)
    assert_maps_equal(gv, ov)
    assert gv["w"].max() == 2000


def test_domain_edge_drops_like_oracle(single):
    """A box that cuts through the scene: returns whose cube leaves it are
    dropped on both sides and cleared samples outside are skipped."""
    W, fr = single
    W2 = workload.Workload(W.name, W.params, W.scene, (11, -2, -2), (4, 3, 3), W.dirs)
    g, o = _both(W2, [(fr.pts, fr.pose)])
    gv, ov = gpu_voxels(g), oracle_voxels(o)
    assert 0 < len(ov["ijk"])
    assert_maps_equal(gv, ov)
    assert g.stats()["returns_accepted"] < len(fr.pts)


def test_deterministic_and_order_independent(single):
    W, fr = single
    perm = np.random.default_rng(3).permutation(len(fr.pts))
    a, _ = _both(W, [(fr.pts, fr.pose)])
    b, _ = _both(W, [(fr.pts[perm], fr.pose)])
    va, vb = gpu_voxels(a), gpu_voxels(b)
    for k in va:
        np.testing.assert_array_equal(va[k], vb[k])


def test_capacity_error_keeps_last_committed_scan(single):
    """A pool too small for the second scan: AF_ERR_CAPACITY is latched, the
    second scan is not integrated, and the map equals the first scan's."""
    W, fr = single
    first = (fr.pts[:200], fr.pose)
    g0, o0 = _both(W, [first])
    need = g0.block_count()
    g, _ = _both(W, [first, (fr.pts, fr.pose)], pool_blocks=need + 5)
    assert g.sync_status() == af.ERR_CAPACITY
    assert_maps_equal(gpu_voxels(g), oracle_voxels(o0))
    with pytest.raises(af.AfError) as e:
        g.frame_host(fr.pts[:10].copy(), fr.pose, np.zeros((0, 3), np.float32),
                     np.zeros((0, 3), np.float32), np.zeros(0, np.uint8),
                     np.zeros(0, np.int16))
    assert e.value.status == 2


def test_too_many_returns_is_rejected(single):
    W, fr = single
    g = gpu_map(W, max_returns=100)
    with pytest.raises(af.AfError) as e:
        g.integrate_scan(to_dev(fr.pts[:101]), fr.pose)
    assert e.value.status == 2
