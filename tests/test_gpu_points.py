"""The stateful point layer on the GPU (af_points_*) against the oracle's
(or_pts_*), frame by frame on the same scans: point ids and voxels, normals,
labels, stored scores and directions, accessibility confidence a, queue
flags and stored viewpoints, all bit for bit -- under a per-frame budget
that leaves a backlog, after draining it, and through the triggers of a
moving sensor and a changing scene. The neighbourhood trigger of Sec. 3.5 is
taken in each of its forms: changed voxels within r_u drawn 256 per frame
(the default), 16 or 1 per frame, all of them, and the brick rule; scenes
where a cleared-band mark alone, or the TSDF move alone, queues points."""
import numpy as np
import pytest

import oracle
from parity import oracle_config, oracle_tool, to_dev
from paper_2608_06412_gb300 import af, synth, workload

pytestmark = pytest.mark.gpu

FIELDS = ("ijk", "normal", "label", "score", "best", "a", "queued", "nviews")


def _compare(g, o, what):
    assert len(g["label"]) == len(o["label"]), (what, len(g["label"]), len(o["label"]))
    for k in FIELDS:
        a, b = g[k], o[k]
        if k in ("normal", "a"):
            a, b = a.view(np.uint32), b.view(np.uint32)      # bit for bit
        bad = np.nonzero((a != b).reshape(len(a), -1).any(1))[0]
        assert len(bad) == 0, f"{what}: {k} differs at {len(bad)} points, first {bad[0]}: " \
                              f"gpu {g[k][bad[0]]} oracle {o[k][bad[0]]}"


def _pair(W, pc, caps, G=None):
    g = af.Map(W.af_config(**caps))
    dirs = W.dirs if G is None else synth.fibonacci_dirs(G)
    g.set_tool(W.af_tool(), dirs)
    g.points_enable(af.PointsConfig(trig_tsdf=2 * W.params["v"], **pc))
    om = oracle.Map(oracle_config(W))
    op = oracle.PointSet(om, oracle.PointsConfig(trig_tsdf=2 * W.params["v"],
                                                 **{k: v for k, v in pc.items() if k != "capacity"}),
                         oracle_tool(W), dirs)
    return g, om, op


TRIGGERS = {"sampled": {}, "sample16": dict(trig_sample=16), "all": dict(trig_sample=0),
            "brick": dict(trig_exact=0)}


@pytest.mark.parametrize("trig", list(TRIGGERS))
def test_points_single_frame_scene_moving_sensor(trig):
    """The sphere / wall / slotted-plate scene from a sensor that moves 4 cm
    per frame: new points, viewpoints, neighbourhood and motion triggers, a
    budget of 150 evaluations per frame, then the backlog drained."""
    W = workload.single_frame()
    caps = dict(hash_capacity=1 << 16, pool_blocks=1 << 14, max_returns=1 << 15, max_points=1 << 12)
    g, om, op = _pair(W, dict(budget=150, capacity=1 << 16, **TRIGGERS[trig]), caps)
    scene = W.scene
    for f in range(8):
        fr = synth.cone_frame(scene, 6000, 0.01, 100 + f, origin=(0.0, 0.04 * f, 0.02 * f))
        g.points_frame(to_dev(fr.pts), fr.pose)
        op.frame(fr.pts, fr.pose)
        _compare(g.points_export(), op.export(), f"frame {f}")
    g.points_drain(10 ** 6)
    op.drain(10 ** 6)
    ge, oe = g.points_export(), op.export()
    _compare(ge, oe, "drained")
    assert (ge["queued"] == 0).all()
    assert (ge["label"] == af.ACCESSIBLE).any() and (ge["label"] == af.BLOCKED).any()
    assert (ge["nviews"] >= 2).any() and (ge["score"] >= 0).mean() > 0.5
    assert g.sync_status() == 0


def test_points_non_default_parameters():
    """Every parameter of the layer away from the paper's value: a 5^3
    neighbour cube with 6 neighbours, 3 viewpoints 5 cm apart, a stricter
    observation filter, a high confidence gate, a faster motion trigger and
    other confidence constants; budget 200."""
    W = workload.single_frame()
    caps = dict(hash_capacity=1 << 16, pool_blocks=1 << 14, max_returns=1 << 15, max_points=1 << 12)
    pc = dict(budget=200, capacity=1 << 16, k_nn=6, nn_radius=2, max_views=3, view_min_dist=0.05,
              obs_dot=0.5, c_min=0.9, k_c=3.0, trig_move=0.05, a_decay=0.5, a_recover=0.3,
              ca_min=0.6)
    g, om, op = _pair(W, pc, caps)
    for f in range(8):
        fr = synth.cone_frame(W.scene, 6000, 0.01, 200 + f, origin=(0.0, 0.03 * f, -0.02 * f))
        g.points_frame(to_dev(fr.pts), fr.pose)
        op.frame(fr.pts, fr.pose)
        _compare(g.points_export(), op.export(), f"frame {f}")
    g.points_drain(10 ** 6)
    op.drain(10 ** 6)
    ge = g.points_export()
    _compare(ge, op.export(), "drained")
    assert ge["nviews"].max() == 3 and (ge["score"] == -1).any() and (ge["score"] >= 0).any()
    assert g.sync_status() == 0


@pytest.mark.parametrize("trig", ["sampled", "brick"])
def test_points_pine_stream(trig):
    """Ten frames of the pine stream (K = 32 directions), 400 evaluations per frame."""
    W = workload.pine_stream()
    caps = dict(hash_capacity=1 << 18, pool_blocks=1 << 16, max_returns=1 << 15, max_points=1 << 12)
    g, om, op = _pair(W, dict(budget=400, capacity=1 << 18, **TRIGGERS[trig]), caps, G=64)
    for f in range(10):
        fr, _, _ = workload.pine_frame(W, f)
        g.points_frame(to_dev(fr.pts), fr.pose)
        op.frame(fr.pts, fr.pose)
    _compare(g.points_export(), op.export(), "frame 9")
    n, ev = g.points_stats()
    assert ev == 400 and n > 10_000
    g.points_drain(2000)
    op.drain(2000)
    _compare(g.points_export(), op.export(), "after a drain of 2000")


def test_points_arguments():
    W = workload.single_frame()
    caps = dict(hash_capacity=1 << 14, pool_blocks=1 << 12, max_returns=1 << 12, max_points=1 << 10)
    g = af.Map(W.af_config(**caps))
    with pytest.raises(af.AfError) as e:
        g.points_frame(to_dev(np.zeros((1, 3), np.float32)), np.eye(4))
    assert e.value.status == af.ERR_STATE
    with pytest.raises(af.AfError) as e:
        g.points_enable(af.PointsConfig(trig_tsdf=0.04, nn_radius=4))
    assert e.value.status == af.ERR_INVALID_ARG
    g.points_enable(af.PointsConfig(trig_tsdf=0.04, capacity=16))
    with pytest.raises(af.AfError) as e:
        g.points_frame(to_dev(np.zeros((1, 3), np.float32)), np.eye(4))
    assert e.value.status == af.ERR_STATE             # no tool yet
    g.set_tool(W.af_tool(), W.dirs)
    fr = synth.cone_frame(W.scene, 500, 0.01, 3)
    g.points_frame(to_dev(fr.pts), fr.pose)          # more points than capacity
    n, _ = g.points_stats()
    assert n == 16 and g.sync_status() == af.ERR_CAPACITY


def _box_workload(boxes, **params):
    """A workload of axis-aligned boxes seen from the origin (v = 2 cm)."""
    g = synth.Group(a=np.array([1.9, 0, 0]), b=np.array([1.9, 0, 0]), radius=0.8,
                    boxes=np.asarray(boxes, np.float64))
    sc = synth.Scene([g], *synth._bounds([g]))
    p = dict(synth.SINGLE_FRAME)
    p.update(params)
    dmin, db = synth.domain_bricks(np.minimum(sc.lo, 0.0), np.maximum(sc.hi, 0.0), p["v"],
                                   margin=0.5)
    return workload.Workload("boxes", p, sc, dmin, db, synth.fibonacci_dirs(64))


def _frames_then_drain(W, pc, frames):
    """Each frame with no evaluation, compared; then both drained, compared."""
    caps = dict(hash_capacity=1 << 16, pool_blocks=1 << 14, max_returns=1 << 15, max_points=1 << 12)
    g, om, op = _pair(W, dict(budget=0, capacity=1 << 16, **pc), caps)
    for f, (pts, pose) in enumerate(frames):
        g.points_frame(to_dev(pts), pose)
        op.frame(pts, pose)
        ge = g.points_export()
        _compare(ge, op.export(), f"frame {f}")
        queued = int(ge["queued"].sum())
        g.points_drain(10 ** 6)
        op.drain(10 ** 6)
        _compare(g.points_export(), op.export(), f"frame {f} drained")
    assert g.sync_status() == 0
    return queued


@pytest.mark.parametrize("trig", ["all", "sampled", "brick"])
def test_points_cleared_band_marks_trigger(trig):
    """A pole 26 cm in front of a wall: the first frame keeps the pole's
    returns, the second the wall's, whose cleared band, stretched to
    (tau, 4 tau], passes beside the pole; the wall's cubes stay more than r_u
    from it. The marks alone re-queue pole points (the brick rule through
    the band samples' bricks)."""
    W = _box_workload([[2.0, -0.3, -0.3, 2.04, 0.3, 0.3], [1.74, -0.04, -0.3, 1.76, 0.04, 0.3]],
                      clear_hi=4.0, clear_samples=12)
    f1 = synth.cone_frame(W.scene, 6000, 0.0, 5)
    f2 = synth.cone_frame(W.scene, 6000, 0.0, 6)
    frames = [(f1.pts[f1.world[:, 0] < 1.9], f1.pose), (f2.pts[f2.world[:, 0] > 1.9], f2.pose)]
    queued = _frames_then_drain(W, TRIGGERS[trig], frames)
    if trig != "sampled":
        assert queued > 10


def test_points_tsdf_trigger_alone():
    """The wall moves 6 cm back and is seen by ten times as many returns: the
    TSDF at its old surface voxels rises by more than 2v, and with one changed
    voxel drawn per frame the TSDF trigger alone queues most of them."""
    W = _box_workload([[2.0, -0.3, -0.3, 2.04, 0.3, 0.3]])
    W2 = _box_workload([[2.06, -0.3, -0.3, 2.10, 0.3, 0.3]])
    f1 = synth.cone_frame(W.scene, 2000, 0.0, 1)
    f2 = synth.cone_frame(W2.scene, 20000, 0.0, 2)
    queued = _frames_then_drain(W, dict(trig_sample=1), [(f1.pts, f1.pose), (f2.pts, f2.pose)])
    assert queued > 50
