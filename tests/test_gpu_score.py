"""GPU parity of accessibility scoring (Sec. 3.4, 3.5) against the oracle:
labels and best-direction indices must be identical when both sides score
the same points against maps integrated from the same scans (integration
parity is checked separately, bit for bit)."""
import numpy as np
import pytest

import oracle
from parity import gpu_map, oracle_config, oracle_tool, to_dev
from paper_2608_06412_gb300 import af, synth, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def single():
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    g = gpu_map(W)
    g.integrate_scan(to_dev(fr.pts), fr.pose)
    o = oracle.Map(oracle_config(W))
    o.integrate(fr.pts, fr.pose)
    return W, fr, pts, nrm, g, o


def _gpu_score(g, pts, nrm):
    import torch
    lab, best = g.score(to_dev(pts.astype(np.float32)), to_dev(nrm.astype(np.float32)))
    torch.cuda.synchronize()
    return lab.cpu().numpy(), best.cpu().numpy()


def _compare(gl, gb, ol, ob):
    bad = np.nonzero((gl != ol) | (gb != ob))[0]
    assert len(bad) == 0, f"{len(bad)} points differ; first {bad[0]}: gpu ({gl[bad[0]]}, " \
                          f"{gb[bad[0]]}) oracle ({ol[bad[0]]}, {ob[bad[0]]})"


def test_single_frame_all_points(single):
    """Every surface point of the single frame (K = 32 of G = 64)."""
    W, fr, pts, nrm, g, o = single
    g.set_tool(W.af_tool(), W.dirs)
    gl, gb = _gpu_score(g, pts, nrm)
    ol, ob = o.score(oracle_tool(W), W.dirs, pts, nrm)
    _compare(gl, gb, ol, ob)
    # the scene exercises both outcomes (every point here is confident)
    for lab in (oracle.ACCESSIBLE, oracle.BLOCKED):
        assert (ol == lab).sum() > 20, lab
    st = g.stats()
    assert st["points_scored"] == int((ol != 0).sum())


def test_strict_corridor_and_narrow_cone(single):
    """Unknown corridor voxels blocking, and the paper's 70 degree normal cone."""
    W, fr, pts, nrm, g, o = single
    sub = slice(0, 1500)
    for over in (dict(strict=1), dict(cos_theta_max=0.342), dict(n_c=1, corr_length=0.5)):
        t = dict(W.tool())
        t.update(over)
        g.set_tool(af.ToolConfig(**t), W.dirs)
        gl, gb = _gpu_score(g, pts[sub], nrm[sub])
        ol, ob = o.score(oracle.Tool(**t), W.dirs, pts[sub], nrm[sub])
        _compare(gl, gb, ol, ob)


def test_edge_points(single):
    """Zero normals (no candidate), points outside the map box, points in
    empty space, a ragged count, and m = 0."""
    W, fr, pts, nrm, g, o = single
    g.set_tool(W.af_tool(), W.dirs)
    p = pts[:37].copy()
    n = nrm[:37].copy()
    n[::5] = 0.0
    p[1] = [100.0, 0.0, 0.0]
    p[2] = [0.5, 0.3, 0.2]
    gl, gb = _gpu_score(g, p, n)
    ol, ob = o.score(oracle_tool(W), W.dirs, p, n)
    _compare(gl, gb, ol, ob)
    assert gl[1] == 0 and gl[2] == 0
    assert ((gl[::5] == 0) | ((gl[::5] == 2) & (gb[::5] == -1))).all()
    gl0, gb0 = _gpu_score(g, p[:0], n[:0])
    assert gl0.shape == (0,)


def test_many_directions(single):
    """G = 512 directions (the large-map orientation count) on a point sample."""
    W, fr, pts, nrm, g, o = single
    dirs = synth.fibonacci_dirs(512)
    g.set_tool(W.af_tool(), dirs)
    sub = slice(0, 400)
    gl, gb = _gpu_score(g, pts[sub], nrm[sub])
    ol, ob = o.score(oracle_tool(W), dirs, pts[sub], nrm[sub])
    _compare(gl, gb, ol, ob)


def test_stream_frame_points():
    """Pine stream: 12 frames integrated, the last frame's points scored (K = 64)."""
    W = workload.pine_stream()
    g = gpu_map(W, hash_capacity=1 << 18, pool_blocks=1 << 17)
    o = oracle.Map(oracle_config(W))
    for f in range(0, 120, 10):
        fr, pts, nrm = workload.pine_frame(W, f)
        g.integrate_scan(to_dev(fr.pts), fr.pose)
        o.integrate(fr.pts, fr.pose)
    g.set_tool(W.af_tool(), W.dirs)
    sel = np.random.default_rng(0).choice(len(pts), 1500, replace=False)
    gl, gb = _gpu_score(g, pts[sel], nrm[sel])
    ol, ob = o.score(oracle_tool(W), W.dirs, pts[sel], nrm[sel])
    _compare(gl, gb, ol, ob)
    assert (ol == oracle.ACCESSIBLE).sum() > 10 and (ol == oracle.BLOCKED).sum() > 10


def test_frame_host_matches_device_path(single):
    """af_frame_host (host buffers, copies inside) = af_integrate_scan + af_score."""
    import torch
    W, fr, pts, nrm, _, _ = single
    a = gpu_map(W)
    a.set_tool(W.af_tool(), W.dirs)
    lab = np.zeros(len(pts), np.uint8)
    best = np.zeros(len(pts), np.int16)
    a.frame_host(np.ascontiguousarray(fr.pts), fr.pose, pts, nrm, lab, best)
    b = gpu_map(W)
    b.set_tool(W.af_tool(), W.dirs)
    b.integrate_scan(to_dev(fr.pts), fr.pose)
    gl, gb = _gpu_score(b, pts, nrm)
    np.testing.assert_array_equal(lab, gl)
    np.testing.assert_array_equal(best, gb)


def test_score_before_tool_is_state_error(single):
    W = single[0]
    g = gpu_map(W)
    with pytest.raises(af.AfError) as e:
        _gpu_score(g, np.zeros((4, 3), np.float32), np.ones((4, 3), np.float32))
    assert e.value.status == af.ERR_STATE


@pytest.fixture(scope="module")
def oracle_single(single):
    W, fr, pts, nrm, g, o = single
    return o.score(oracle_tool(W), W.dirs, pts, nrm)


@pytest.mark.parametrize("budget", [-1, 0, 1, 3, 8, 1000])
def test_work_sharing_budgets(single, oracle_single, budget):
    """af_set_score_split: every hand-off threshold gives the single-pass
    result (0: every searched direction is its own warp; -1: no hand-off)."""
    W, fr, pts, nrm, g, o = single
    g.set_tool(W.af_tool(), W.dirs)
    g.set_score_split(budget)
    try:
        gl, gb = _gpu_score(g, pts, nrm)
    finally:
        g.set_score_split(-1)
    _compare(gl, gb, *oracle_single)


def test_work_sharing_grows_past_max_points(single, oracle_single):
    """More points per call than the map's max_points: the hand-off records
    grow; a bad budget is rejected."""
    W, fr, pts, nrm, _, o = single
    g = gpu_map(W, max_points=64)
    g.integrate_scan(to_dev(fr.pts), fr.pose)
    g.set_tool(W.af_tool(), W.dirs)
    g.set_score_split(0)
    gl, gb = _gpu_score(g, pts, nrm)
    _compare(gl, gb, *oracle_single)
    with pytest.raises(af.AfError) as e:
        g.set_score_split(-2)
    assert e.value.status == af.ERR_INVALID_ARG


def test_work_sharing_pine_frames():
    """The hand-off (budget 4) on pine-stream frames, whose points are heavier
    and more uneven than the single frame's: labels and directions equal the
    single-pass search on the same map."""
    import torch
    W = workload.pine_stream()
    g = gpu_map(W, hash_capacity=1 << 18, pool_blocks=1 << 16, max_returns=1 << 15)
    g.set_tool(W.af_tool(), W.dirs)
    for f in range(12):
        fr, pts, nrm = workload.pine_frame(W, f)
        g.integrate_scan(to_dev(fr.pts), fr.pose)
    g.set_score_split(-1)
    a = _gpu_score(g, pts, nrm)
    g.set_score_split(4)
    b = _gpu_score(g, pts, nrm)
    g.set_score_split(-1)
    _compare(*b, *a)
    assert (a[0] == af.ACCESSIBLE).sum() > 100 and (a[0] == af.BLOCKED).sum() > 100


def test_points_near_the_box_faces():
    """A map box barely larger than the scene and smaller than twice the
    kernels' reach (corridor 1 m = 50 voxels): every scored point takes the
    bounds-checked path, with runs along all three axes reading voxels beyond
    the faces as free and unknown."""
    import torch
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    W2 = workload.Workload(W.name, W.params, W.scene, (9, -4, -5), (8, 8, 10), W.dirs)
    g = gpu_map(W2)
    g.integrate_scan(to_dev(fr.pts), fr.pose)
    o = oracle.Map(oracle_config(W2))
    o.integrate(fr.pts, fr.pose)
    g.set_tool(W.af_tool(), W.dirs)
    gl, gb = _gpu_score(g, pts, nrm)
    ol, ob = o.score(oracle_tool(W), W.dirs, pts, nrm)
    _compare(gl, gb, ol, ob)
    assert (ol == oracle.ACCESSIBLE).sum() > 20 and (ol == oracle.BLOCKED).sum() > 20
