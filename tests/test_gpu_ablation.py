"""The paper's variants and ablations on the GPU against the oracle.

* The [-tau, tau] clamp of Tab. 4 (the map's `clamp_signed`): maps bit for
  bit, including a weight cap of 3 whose rescale of negative sums rounds
  toward minus infinity; labels and best directions, the soft clearance and
  the stateful layer on such a map.
* The paper's approach set (Sec. 3.4): the 180-direction horizontal yaw ring
  with the 70 degree normal cone, in the plain scorer and the stateful layer.
* The coarse-to-fine search of Sec. 3.6 (20 degree coarse stride, +-24
  degree window around the nearest resolved neighbour's direction within
  0.3 m) in the stateful layer, frame by frame and after draining.
* Projective integration, the ablation of Tab. 3: maps bit for bit over an
  octahedral range image, single scans and a rotating stream, both clamps,
  and labels on the projective map.
"""
import numpy as np
import pytest

import oracle
from parity import (assert_maps_equal, gpu_map, gpu_voxels, oracle_config, oracle_tool,
                    oracle_voxels, to_dev)
from paper_2608_06412_gb300 import af, synth, workload

pytestmark = pytest.mark.gpu

PINE_CAPS = dict(hash_capacity=1 << 18, pool_blocks=1 << 16, max_returns=1 << 15,
                 max_points=1 << 15)


@pytest.fixture(scope="module")
def signed_single():
    import torch
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    g = gpu_map(W, clamp_signed=1)
    g.integrate_scan(to_dev(fr.pts), fr.pose)
    o = oracle.Map(oracle_config(W, clamp_signed=1))
    o.integrate(fr.pts, fr.pose)
    torch.cuda.synchronize()
    return W, fr, pts, nrm, g, o


def test_signed_clamp_single_frame_bit_exact(signed_single):
    W, fr, pts, nrm, g, o = signed_single
    assert g.sync_status() == 0
    gv, ov = gpu_voxels(g), oracle_voxels(o)
    assert_maps_equal(gv, ov)
    assert (gv["S"] < 0).sum() > 1000 and (gv["S"] > 0).sum() > 1000


def test_signed_clamp_stream_with_cap_bit_exact():
    """Ten pine-stream frames with w_cap = 3: the cap rescales negative sums
    on every scan."""
    import torch
    W = workload.pine_stream()
    g = gpu_map(W, clamp_signed=1, w_cap=3, **PINE_CAPS)
    o = oracle.Map(oracle_config(W, clamp_signed=1, w_cap=3))
    for f in range(10):
        fr, _, _ = workload.pine_frame(W, f)
        g.integrate_scan(to_dev(fr.pts), fr.pose)
        o.integrate(fr.pts, fr.pose)
    torch.cuda.synchronize()
    assert g.sync_status() == 0
    gv = gpu_voxels(g)
    assert_maps_equal(gv, oracle_voxels(o))
    neg = gv["S"] < 0
    assert neg.sum() > 1000 and (gv["w"][neg] == 3).sum() > 100


def test_signed_clamp_labels(signed_single):
    import torch
    W, fr, pts, nrm, g, o = signed_single
    g.set_tool(W.af_tool(), W.dirs)
    lab, best = g.score(to_dev(pts.astype(np.float32)), to_dev(nrm.astype(np.float32)))
    torch.cuda.synchronize()
    ol, ob = o.score(oracle_tool(W), W.dirs, pts, nrm)
    gl, gb = lab.cpu().numpy(), best.cpu().numpy()
    bad = np.nonzero((gl != ol) | (gb != ob))[0]
    assert len(bad) == 0, (len(bad), bad[:5])
    assert (ol == oracle.ACCESSIBLE).sum() > 20 and (ol == oracle.BLOCKED).sum() > 20


def test_signed_clamp_soft_clearance(signed_single):
    """Negative voxel TSDFs reach the soft clearance through the dense view."""
    import torch
    W, fr, pts, nrm, g, o = signed_single
    g.set_tool(W.af_tool(), W.dirs)
    rng = np.random.default_rng(5)
    idx = rng.choice(len(pts), 200, replace=False)
    P, N = pts[idx], nrm[idx]
    K = 8
    u0 = oracle.soft_seed(N, synth.fibonacci_hemisphere(K))
    n = len(u0)
    al = rng.uniform(-0.3, 0.3, n).astype(np.float32)
    be = rng.uniform(-0.3, 0.3, n).astype(np.float32)
    h = rng.uniform(0.0, 0.03, n).astype(np.float32)
    cmin = torch.empty(n, dtype=torch.float32, device="cuda")
    f = lambda x: to_dev(np.ascontiguousarray(x, np.float32))
    c = g.soft_clearance_raw(f(P), f(u0), f(al), f(be), f(h), K, 0.005, cmin=cmin).cpu().numpy()
    ref, _ = o.soft_clearance(oracle_tool(W), P, K, u0, al, be, h, 0.005)
    np.testing.assert_allclose(c, ref, rtol=0, atol=1e-5)
    np.testing.assert_allclose(cmin.cpu().numpy(), o.last_cmin, rtol=0, atol=1e-5)
    assert (o.last_cmin < -0.05).any()       # a sample reads a negative voxel


def test_signed_clamp_point_layer():
    """The stateful layer reads w and the TSDF of a signed map."""
    W = workload.single_frame()
    caps = dict(hash_capacity=1 << 16, pool_blocks=1 << 14, max_returns=1 << 15, max_points=1 << 12)
    g = af.Map(W.af_config(clamp_signed=1, **caps))
    g.set_tool(W.af_tool(), W.dirs)
    v = W.params["v"]
    g.points_enable(af.PointsConfig(trig_tsdf=2 * v, budget=300, capacity=1 << 16))
    om = oracle.Map(oracle_config(W, clamp_signed=1))
    op = oracle.PointSet(om, oracle.PointsConfig(trig_tsdf=2 * v, budget=300), oracle_tool(W),
                         W.dirs)
    for k in range(5):
        fr = synth.cone_frame(W.scene, 6000, 0.01, 300 + k, origin=(0.0, -0.05 * k, 0.03 * k))
        g.points_frame(to_dev(fr.pts), fr.pose)
        op.frame(fr.pts, fr.pose)
    ge, oe = g.points_export(), op.export()
    for key in ("ijk", "normal", "label", "score", "best", "a", "queued", "nviews"):
        a, b = ge[key], oe[key]
        if key in ("normal", "a"):
            a, b = a.view(np.uint32), b.view(np.uint32)
        assert (a == b).all(), key
    assert g.sync_status() == 0


FIELDS = ("ijk", "normal", "label", "score", "best", "a", "queued", "nviews")


def _same_points(ge, oe, what):
    assert len(ge["label"]) == len(oe["label"]), what
    for key in FIELDS:
        a, b = ge[key], oe[key]
        if key in ("normal", "a"):
            a, b = a.view(np.uint32), b.view(np.uint32)
        bad = np.nonzero((a != b).reshape(len(a), -1).any(1))[0]
        assert len(bad) == 0, f"{what}: {key} differs at {len(bad)} points, first {bad[0]}"


def _ring_tool(W):
    t = dict(W.tool())
    t["cos_theta_max"] = synth.COS_70
    return t


def test_yaw_ring_scoring():
    """The plain scorer over the yaw ring (G = 180, not a multiple of 32)."""
    import torch
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    g = gpu_map(W)
    g.integrate_scan(to_dev(fr.pts), fr.pose)
    o = oracle.Map(oracle_config(W))
    o.integrate(fr.pts, fr.pose)
    dirs = synth.yaw_ring(180)
    t = _ring_tool(W)
    g.set_tool(af.ToolConfig(**t), dirs)
    lab, best = g.score(to_dev(pts.astype(np.float32)), to_dev(nrm.astype(np.float32)))
    torch.cuda.synchronize()
    ol, ob, ds = o.score(oracle.Tool(**t), dirs, pts, nrm, dir_scores=True)
    gl, gb = lab.cpu().numpy(), best.cpu().numpy()
    bad = np.nonzero((gl != ol) | (gb != ob))[0]
    assert len(bad) == 0, (len(bad), bad[:5])
    assert (ol == oracle.ACCESSIBLE).sum() > 20 and (ol == oracle.BLOCKED).sum() > 20
    assert (ds[:, 160:] >= 0).any()   # the last, partial group of 32 holds candidates


@pytest.mark.parametrize("c2f", [False, True])
def test_yaw_ring_point_layer(c2f):
    """The stateful layer on the yaw ring, with and without the coarse-to-fine
    search: a moving sensor, 250 evaluations per frame, then a full drain."""
    W = workload.single_frame()
    caps = dict(hash_capacity=1 << 16, pool_blocks=1 << 14, max_returns=1 << 15, max_points=1 << 12)
    dirs = synth.yaw_ring(180)
    t = _ring_tool(W)
    extra = dict(c2f_stride=10, c2f_half=12, c2f_radius=0.3) if c2f else {}
    v = W.params["v"]
    g = af.Map(W.af_config(**caps))
    g.set_tool(af.ToolConfig(**t), dirs)
    g.points_enable(af.PointsConfig(trig_tsdf=2 * v, budget=250, capacity=1 << 16, **extra))
    om = oracle.Map(oracle_config(W))
    op = oracle.PointSet(om, oracle.PointsConfig(trig_tsdf=2 * v, budget=250, **extra),
                         oracle.Tool(**t), dirs)
    for k in range(6):
        fr = synth.cone_frame(W.scene, 6000, 0.01, 400 + k, origin=(0.0, 0.04 * k, 0.0))
        g.points_frame(to_dev(fr.pts), fr.pose)
        op.frame(fr.pts, fr.pose)
        _same_points(g.points_export(), op.export(), f"frame {k}")
    g.points_drain(10 ** 6)
    op.drain(10 ** 6)
    ge = g.points_export()
    _same_points(ge, op.export(), "drained")
    assert (ge["label"] == af.ACCESSIBLE).sum() > 50 and (ge["label"] == af.BLOCKED).sum() > 50
    assert g.sync_status() == 0


def test_coarse_to_fine_pine_stream():
    """Eight pine-stream frames on the yaw ring with the coarse-to-fine search."""
    W = workload.pine_stream()
    dirs = synth.yaw_ring(180)
    t = _ring_tool(W)
    extra = dict(c2f_stride=10, c2f_half=12, c2f_radius=0.3)
    v = W.params["v"]
    g = af.Map(W.af_config(**PINE_CAPS))
    g.set_tool(af.ToolConfig(**t), dirs)
    g.points_enable(af.PointsConfig(trig_tsdf=2 * v, budget=600, capacity=1 << 18, **extra))
    om = oracle.Map(oracle_config(W))
    op = oracle.PointSet(om, oracle.PointsConfig(trig_tsdf=2 * v, budget=600, **extra),
                         oracle.Tool(**t), dirs)
    for f in range(8):
        fr, _, _ = workload.pine_frame(W, f)
        g.points_frame(to_dev(fr.pts), fr.pose)
        op.frame(fr.pts, fr.pose)
    _same_points(g.points_export(), op.export(), "frame 7")
    g.points_drain(3000)
    op.drain(3000)
    ge = g.points_export()
    _same_points(ge, op.export(), "after a drain of 3000")
    assert (ge["best"] >= 0).sum() > 1000


@pytest.mark.parametrize("clamp_signed,bins", [(0, 812), (1, 812), (0, 97)])
def test_projective_single_frame_bit_exact(clamp_signed, bins):
    import torch
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    g = gpu_map(W, clamp_signed=clamp_signed)
    g.integrate_scan_projective(to_dev(fr.pts), fr.pose, bins)
    o = oracle.Map(oracle_config(W, clamp_signed=clamp_signed))
    o.integrate_projective(fr.pts, fr.pose, bins)
    torch.cuda.synchronize()
    assert g.sync_status() == 0
    gv = gpu_voxels(g)
    assert_maps_equal(gv, oracle_voxels(o))
    assert len(gv["w"]) > 10000 and (gv["cleared"] == 0).all()


def test_projective_stream_and_labels():
    """Eight pine-stream frames (the sensor orbits, so every pose rotates),
    then scoring on the projective map."""
    import torch
    W = workload.pine_stream()
    g = gpu_map(W, **PINE_CAPS)
    o = oracle.Map(oracle_config(W))
    for f in range(8):
        fr, pts, nrm = workload.pine_frame(W, f)
        g.integrate_scan_projective(to_dev(fr.pts), fr.pose)
        o.integrate_projective(fr.pts, fr.pose)
    torch.cuda.synchronize()
    assert g.sync_status() == 0
    assert_maps_equal(gpu_voxels(g), oracle_voxels(o))
    g.set_tool(W.af_tool(), W.dirs)
    sel = np.random.default_rng(3).choice(len(pts), min(2000, len(pts)), replace=False)
    lab, best = g.score(to_dev(pts[sel].astype(np.float32)), to_dev(nrm[sel].astype(np.float32)))
    torch.cuda.synchronize()
    ol, ob = o.score(oracle_tool(W), W.dirs, pts[sel], nrm[sel])
    assert (lab.cpu().numpy() == ol).all() and (best.cpu().numpy() == ob).all()


def test_projective_arguments():
    W = workload.single_frame()
    g = gpu_map(W)
    with pytest.raises(af.AfError) as e:
        g.integrate_scan_projective(to_dev(np.zeros((4, 3), np.float32)), np.eye(4), 1)
    assert e.value.status == af.ERR_INVALID_ARG
    g.integrate_scan_projective(to_dev(np.zeros((0, 3), np.float32)), np.eye(4), 64)
    assert g.sync_status() == 0 and len(gpu_voxels(g)["w"]) == 0
