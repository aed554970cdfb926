"""Pins of the oracle's stateful layer (Sec. 3.4 normals and observation-side
filter, Sec. 3.5 incremental updates and confidence) against what the paper
and mathematics fix:

* the Jacobi eigen-solver against numpy's LAPACK solver, residuals and
  orthonormality, and the diagonal case (no rotation at all);
* normals on a voxelised sphere against a brute-force restatement (nearest
  neighbours by sorting, float64 covariance, numpy's eigen-solver);
* PCA normals on an axis-aligned wall equal the wall normal exactly, facing
  the sensor; points are numbered in (z, y, x) order within a frame;
* viewpoints are stored only when farther than the minimum distance from all
  stored ones, at most max_views (8, and 3 when configured so);
* the confidence gate skips exactly the points with w / (w + k_c) < c_min;
* every scored best direction is aligned (> obs_dot) with a stored viewpoint;
* the budget evaluates the lowest ids first and the backlog drains in order;
* the paper's worked example: a well-observed accessible point stays
  accessible after one conflicting evaluation (c a = 0.75) and leaves the
  accessible set after two (c a = 0.5625 < 0.7), its stored score unchanged;
* a sensor move above trig_move re-queues blocked points, a smaller one
  does not, and the distance is measured from where the trigger last fired;
  returns far away queue nothing;
* the neighbourhood trigger (a changed voxel within r_u = 3v, among the
  changed voxels drawn for the frame, or all of them) against a brute force
  over the map's voxel states before and after the frame; the TSDF trigger
  firing on its own; the brick rule covering the unsampled voxel rule, which
  covers the sampled one; the hash that draws the sample against published
  splitmix64 outputs;
* the coarse-to-fine search (Sec. 3.6) against a brute force over the plain
  scorer's per-direction scores, for first evaluations and re-evaluations,
  and its degenerate cases against the full search.
Parity status: pinned.
"""
import numpy as np
import pytest

import oracle
from paper_2608_06412_gb300 import synth

V = 0.02


def _cfg():
    return oracle.Config(v=V, tau=0.06, r_c=0.01, cube_radius=3, clear_samples=8,
                         dom_min=(-64, -64, -64), dom_size=(256, 128, 128), w_min=1)


def _tool(**kw):
    base = dict(radius=0.04, length=0.25, self_excl=0.04, corr_radius=0.05, corr_length=0.5,
                cos_theta_max=0.0, n_c=5, strict=0)
    base.update(kw)
    return oracle.Tool(**base)


def _wall(x0=2.0, half=0.5):
    g = synth.Group(a=np.array([x0 + 0.02, 0, -half]), b=np.array([x0 + 0.02, 0, half]),
                    radius=half * 1.5, boxes=np.array([[x0, -half, -half, x0 + 0.04, half, half]]))
    return synth.Scene([g], *synth._bounds([g]))


def _frame(scene, origin, n=4000, seed=0):
    fr = synth.cone_frame(scene, n, 0.0, seed, origin=origin)
    return fr.pts, fr.pose


def test_jacobi_matches_lapack():
    rng = np.random.default_rng(0)
    for k in range(300):
        if k % 3 == 0:   # integer covariance-like matrices, as the normal forms them
            d = rng.integers(-3, 4, (10, 3))
            A = (10 * d.T @ d - np.outer(d.sum(0), d.sum(0))).astype(np.float32)
        else:
            B = rng.normal(size=(3, 3))
            A = (B + B.T).astype(np.float32)
        ev, Vm = oracle.jacobi3(A)
        ref = np.linalg.eigvalsh(A.astype(np.float64))
        scale = max(np.abs(ref).max(), 1e-6)
        np.testing.assert_allclose(np.sort(ev), ref, atol=3e-6 * scale)
        Vd = Vm.astype(np.float64)
        np.testing.assert_allclose(Vd.T @ Vd, np.eye(3), atol=2e-6)
        np.testing.assert_allclose(A @ Vd, Vd * ev, atol=2e-5 * scale)
    A = np.diag([3.0, 1.0, 2.0]).astype(np.float32)
    ev, Vm = oracle.jacobi3(A)
    assert (Vm == np.eye(3)).all() and (ev == [3, 1, 2]).all()


def test_wall_normals_ids_and_views():
    mp = oracle.Map(_cfg())
    P = oracle.PointSet(mp, oracle.PointsConfig(trig_tsdf=2 * V), _tool(), synth.fibonacci_dirs(64))
    pts, pose = _frame(_wall(), (0.0, 0.0, 0.0))
    P.frame(pts, pose)
    e = P.export()
    # ids in (z, y, x) order of the voxels
    order = np.lexsort((e["ijk"][:, 0], e["ijk"][:, 1], e["ijk"][:, 2]))
    assert (order == np.arange(len(order))).all()
    # interior wall points: exactly the -x normal, facing the sensor at x < 2
    scored = e["score"] >= 0
    interior = scored & (np.abs(e["ijk"][:, 1]) < 20) & (np.abs(e["ijk"][:, 2]) < 20)
    assert interior.sum() > 50
    assert (e["normal"][interior] == np.array([-1, 0, 0], np.float32)).all()
    # one scan, one viewpoint each
    assert (e["nviews"] == 1).all()


def _sphere(c=(1.5, 0.0, 0.0), r=0.3):
    c = np.asarray(c, float)
    g = synth.Group(a=c, b=c, radius=r * 1.01, spheres=np.array([[*c, r]]))
    return synth.Scene([g], *synth._bounds([g]))


def test_pca_normals_match_brute_force_eigh():
    """Normals on a voxelised sphere against a brute-force restatement: the 10
    nearest points of the final set in the +-3 cube (ties by dz, dy, dx), the
    covariance in float64 and numpy's symmetric eigen-solver, the smallest
    eigenvector turned toward the sensor."""
    mp = oracle.Map(_cfg())
    P = oracle.PointSet(mp, oracle.PointsConfig(trig_tsdf=2 * V), _tool(), synth.fibonacci_dirs(64))
    origin = np.zeros(3)
    pts, pose = _frame(_sphere(), origin, n=6000)
    P.frame(pts, pose)
    e = P.export()
    ijk = e["ijk"].astype(np.int64)
    keys = {tuple(x): i for i, x in enumerate(ijk)}
    R = 3
    offs = [(x, y, z) for z in range(-R, R + 1) for y in range(-R, R + 1) for x in range(-R, R + 1)]
    offs.sort(key=lambda o: (o[0] ** 2 + o[1] ** 2 + o[2] ** 2, o[2], o[1], o[0]))
    checked = 0
    for i in np.flatnonzero(e["score"] >= 0):
        nb = [o for o in offs if tuple(ijk[i] + o) in keys][:10]
        d = np.array(nb, np.float64)
        C = (d - d.mean(0)).T @ (d - d.mean(0))
        w, Vm = np.linalg.eigh(C)
        if (w[1] - w[0]) < 0.05 * w[2]:
            continue   # near-degenerate smallest pair: the direction is ill-posed
        n = Vm[:, 0]
        s = (ijk[i] + 0.5) * V
        if n @ (origin - s) < 0:
            n = -n
        assert np.abs(e["normal"][i] - n).max() < 2e-4, (i, e["normal"][i], n)
        checked += 1
    assert checked > 200


def test_view_storage_rule():
    mp = oracle.Map(_cfg())
    P = oracle.PointSet(mp, oracle.PointsConfig(trig_tsdf=2 * V, budget=0), _tool(),
                        synth.fibonacci_dirs(32))
    wall = _wall()
    for k in range(20):   # sensor steps of 6 cm: every second position is stored
        pts, pose = _frame(wall, (0.0, 0.06 * k, 0.0), n=3000, seed=k)
        P.frame(pts, pose)
    e = P.export()
    seen_all = e["nviews"][(np.abs(e["ijk"][:, 1]) < 5) & (np.abs(e["ijk"][:, 2]) < 5)]
    assert seen_all.max() == 8            # capped at max_views
    P2 = oracle.PointSet(oracle.Map(_cfg()), oracle.PointsConfig(trig_tsdf=2 * V, budget=0),
                         _tool(), synth.fibonacci_dirs(32))
    for k in range(5):    # positions 0, 6, 12, 18, 24 cm: stored 0, 12, 24
        pts, pose = _frame(wall, (0.0, 0.06 * k, 0.0), n=3000, seed=k)
        P2.frame(pts, pose)
    e2 = P2.export()
    # greedy storage: any two stored positions are > 10 cm apart, so at most
    # 3 of these 5 (storing every scan would give 5, a reversed test 1)
    assert e2["nviews"].max() == 3 and (e2["nviews"] == 3).sum() > 20
    # max_views = 3 with more positions far apart: exactly 3 are kept
    P3 = oracle.PointSet(oracle.Map(_cfg()),
                         oracle.PointsConfig(trig_tsdf=2 * V, budget=0, max_views=3), _tool(),
                         synth.fibonacci_dirs(32))
    for k in range(6):    # 0, 12, ..., 60 cm: six storable positions
        pts, pose = _frame(wall, (0.0, 0.12 * k, 0.0), n=3000, seed=k)
        P3.frame(pts, pose)
    e3 = P3.export()
    assert e3["nviews"].max() == 3 and (e3["nviews"] == 3).sum() > 20


def test_observation_side_filter():
    mp = oracle.Map(_cfg())
    dirs = synth.fibonacci_dirs(128)
    P = oracle.PointSet(mp, oracle.PointsConfig(trig_tsdf=2 * V), _tool(cos_theta_max=-1.0), dirs)
    pts, pose = _frame(_wall(), (0.0, 0.4, 0.0))
    P.frame(pts, pose)
    e = P.export()
    s = (e["ijk"] + 0.5) * np.float32(V)
    ok = e["best"] >= 0
    assert ok.sum() > 50
    to_q = np.array([0.0, 0.4, 0.0]) - s[ok]
    to_q /= np.linalg.norm(to_q, axis=1, keepdims=True)
    assert ((dirs[e["best"][ok]] * to_q).sum(1) > 0.25).all()
    # without the filter some best directions point away from the sensor side
    P2 = oracle.PointSet(oracle.Map(_cfg()), oracle.PointsConfig(trig_tsdf=2 * V, obs_dot=-2.0),
                         _tool(cos_theta_max=-1.0), dirs)
    P2.frame(pts, pose)
    e2 = P2.export()
    ok2 = e2["best"] >= 0
    to_q2 = np.array([0.0, 0.4, 0.0]) - s[ok2]
    to_q2 /= np.linalg.norm(to_q2, axis=1, keepdims=True)
    assert ((dirs[e2["best"][ok2]] * to_q2).sum(1) <= 0.25).any()


def test_budget_and_backlog_in_id_order():
    mp = oracle.Map(_cfg())
    P = oracle.PointSet(mp, oracle.PointsConfig(trig_tsdf=2 * V, budget=7), _tool(),
                        synth.fibonacci_dirs(32))
    pts, pose = _frame(_wall(), (0.0, 0.0, 0.0))
    assert P.frame(pts, pose) == 7
    e = P.export()
    assert (e["queued"][:7] == 0).all() and (e["queued"][7:] == 1).all()
    assert P.drain(10) == 10
    e = P.export()
    assert (e["queued"][:17] == 0).all() and (e["queued"][17:] == 1).all()
    assert P.drain(10 ** 9) == len(P) - 17
    assert P.drain(5) == 0


def test_two_conflicts_leave_the_accessible_set():
    """Sec. 3.5: for a well-observed point (c ~ 1) one conflicting evaluation
    leaves it accessible, two push c a below 0.7; the stored score stays."""
    mp = oracle.Map(_cfg())
    dirs = np.array([[-1.0, 0.0, 0.0]], np.float32)     # one approach direction: from -x
    # every changed voxel is tested (no sample), so the wall's own returns
    # re-queue the point each frame and both blocking evaluations happen
    P = oracle.PointSet(mp, oracle.PointsConfig(trig_tsdf=2 * V, k_c=1e-3, trig_sample=0), _tool(),
                        dirs)
    wall = _wall(half=0.3)
    for k in range(3):
        pts, pose = _frame(wall, (0.0, 0.0, 0.0), n=4000, seed=k)
        P.frame(pts, pose)
    e = P.export()
    centre = np.nonzero((e["ijk"][:, 1] == 0) & (e["ijk"][:, 2] == 0) & (e["score"] >= 0))[0]
    assert len(centre) == 1
    c0 = centre[0]
    assert e["label"][c0] == oracle.ACCESSIBLE and e["score"][c0] < 5 and e["a"][c0] == 1.0
    # an obstacle appears in the corridor (a plate 40 cm in front of the wall)
    plate = synth.Group(a=np.array([1.7, 0, 0]), b=np.array([1.7, 0, 0]), radius=0.2,
                        boxes=np.array([[1.68, -0.1, -0.1, 1.72, 0.1, 0.1]]))
    both = synth.Scene(wall.groups + [plate], *synth._bounds(wall.groups + [plate]))
    labels, a = [], []
    for k in range(2):
        pts, pose = _frame(both, (0.0, 0.0, 0.0), n=4000, seed=10 + k)
        P.frame(pts, pose)
        e = P.export()
        labels.append(int(e["label"][c0]))
        a.append(float(e["a"][c0]))
    assert a == [np.float32(0.75), np.float32(np.float32(0.75) * np.float32(0.75))]
    assert labels == [oracle.ACCESSIBLE, oracle.BLOCKED]
    assert e["score"][c0] < 5              # the stored score never increases


def test_motion_trigger_and_locality():
    """Budget 0: frames only queue; drains evaluate."""
    dirs = synth.fibonacci_dirs(64)
    P = oracle.PointSet(oracle.Map(_cfg()), oracle.PointsConfig(trig_tsdf=2 * V, budget=0),
                        _tool(corr_length=1.0), dirs)
    # a wall with a slot too narrow for the tool, and a second wall behind it
    g = synth.Group(a=np.array([2.02, 0, 0]), b=np.array([2.02, 0, 0]), radius=0.8,
                    boxes=np.array([[2.0, -0.5, -0.5, 2.04, -0.01, 0.5],
                                    [2.0, 0.01, -0.5, 2.04, 0.5, 0.5],
                                    [2.3, -0.5, -0.5, 2.34, 0.5, 0.5]]))
    scene = synth.Scene([g], *synth._bounds([g]))
    pts, pose = _frame(scene, (0.0, 0.0, 0.0), n=6000)
    assert P.frame(pts, pose) == 0
    n0 = len(P)
    assert (P.export()["queued"] == 1).all()          # new points are always queued
    P.drain(10 ** 9)
    e = P.export()
    blocked = e["label"] == oracle.BLOCKED
    assert blocked.any() and (e["label"] == oracle.ACCESSIBLE).any() and (e["queued"] == 0).all()
    # returns 1.2 m aside only, the sensor moved 3 cm: nothing near the wall is queued
    far = synth.Group(a=np.array([0.5, 1.2, 0]), b=np.array([0.5, 1.2, 0]), radius=0.2,
                      boxes=np.array([[0.48, 1.1, -0.1, 0.52, 1.3, 0.1]]))
    sfar = synth.Scene([far], *synth._bounds([far]))
    pts, pose = _frame(sfar, (0.0, 0.03, 0.0), n=500)
    P.frame(pts, pose)
    assert (P.export()["queued"][:n0] == 0).all()
    # 12 cm from where the motion trigger last fired: exactly the blocked points
    pts, pose = _frame(sfar, (0.0, 0.12, 0.0), n=500, seed=1)
    P.frame(pts, pose)
    q = P.export()["queued"][:n0].astype(bool)
    assert (q == blocked).all()
    # 17 cm from the start but 5 cm from the last firing: nothing is re-queued
    P.drain(10 ** 9)
    pts, pose = _frame(sfar, (0.0, 0.17, 0.0), n=500, seed=2)
    P.frame(pts, pose)
    assert (P.export()["queued"][:n0] == 0).all()


def test_state_update_rules():
    """Sec. 3.5 in closed form: the stored score only decreases; a decays by
    0.75 on each conflict and recovers by 0.15 (1 - a) on each confirmation;
    confident-accessible iff stored score < n_c and c a > 0.7."""
    pc = oracle.PointsConfig(trig_tsdf=0.04)
    f = np.float32
    st = dict(score=-1, best=-1, a=1.0)
    st = oracle.pts_state_step(pc, 5, st, 3, 7, 0.99)         # first evaluation
    assert st == dict(score=3, best=7, a=1.0, label=oracle.ACCESSIBLE)
    st = oracle.pts_state_step(pc, 5, st, 5, 2, 0.99)         # s = n_c: a conflict
    assert (st["score"], st["best"], st["a"]) == (3, 7, f(0.75)) and st["label"] == oracle.ACCESSIBLE
    st = oracle.pts_state_step(pc, 5, st, 6, 2, 0.99)         # blocked: a second conflict
    a2 = f(f(0.75) * f(0.75))
    assert st["a"] == a2 and st["label"] == oracle.BLOCKED    # 0.99 * 0.5625 < 0.7
    st = oracle.pts_state_step(pc, 5, st, 1, 4, 0.99)         # confirming, strictly lower
    a3 = f(a2 + f(f(0.15) * f(f(1.0) - a2)))
    assert (st["score"], st["best"], st["a"]) == (1, 4, a3)
    st = oracle.pts_state_step(pc, 5, st, 1, 9, 0.99)         # equal score keeps the direction
    assert st["best"] == 4
    # a point never accessible: scores n_c and above neither decay nor recover a
    st = oracle.pts_state_step(pc, 5, dict(score=-1, best=-1, a=1.0), 5, 0, 1.0)
    assert (st["score"], st["a"], st["label"]) == (5, 1.0, oracle.BLOCKED)
    st = oracle.pts_state_step(pc, 5, st, 6, 1, 1.0)
    assert (st["score"], st["a"], st["label"]) == (5, 1.0, oracle.BLOCKED)
    # one conflict at c = 0.9 already drops c a below 0.7 (0.675)
    st = oracle.pts_state_step(pc, 5, dict(score=2, best=1, a=1.0), 6, 0, 0.9)
    assert st["label"] == oracle.BLOCKED and st["score"] == 2
    # low confidence keeps an accessible score unconfident
    st = oracle.pts_state_step(pc, 5, dict(score=-1, best=-1, a=1.0), 0, 3, 0.6)
    assert st["label"] == oracle.BLOCKED and st["score"] == 0


def test_neighbour_brick_trigger_and_confidence_gate():
    dirs = synth.fibonacci_dirs(32)
    P = oracle.PointSet(oracle.Map(_cfg()), oracle.PointsConfig(trig_tsdf=2 * V, budget=0),
                        _tool(), dirs)
    pts, pose = _frame(_wall(), (0.0, 0.0, 0.0), n=6000)
    P.frame(pts, pose)
    P.drain(10 ** 9)
    n0 = len(P)
    # returns from a small box above the wall's top edge (z voxels 27..29)
    top = synth.Group(a=np.array([2.02, 0, 0.57]), b=np.array([2.02, 0, 0.57]), radius=0.1,
                      boxes=np.array([[2.0, -0.05, 0.55, 2.04, 0.05, 0.59]]))
    st = synth.Scene([top], *synth._bounds([top]))
    pts, pose = _frame(st, (0.0, 0.0, 0.0), n=300)
    P.frame(pts, pose)
    e = P.export()
    old = np.arange(len(e["queued"])) < n0
    zb = np.floor_divide(e["ijk"][:, 2], 8)
    q = e["queued"].astype(bool)
    assert (q & old & (zb == 2)).any()             # one brick below the touched bricks
    assert not (q & old & (zb <= 1)).any()         # two bricks away: untouched
    # a sparse scan: isolated returns leave w = 1 (c = 1/6 < 0.2): never scored, not queued
    P2 = oracle.PointSet(oracle.Map(_cfg()), oracle.PointsConfig(trig_tsdf=2 * V), _tool(), dirs)
    pts, pose = _frame(_wall(), (0.0, 0.0, 0.0), n=25, seed=3)
    P2.frame(pts, pose)
    e2 = P2.export()
    assert len(e2["score"]) >= 20 and (e2["queued"] == 0).all()
    assert (e2["score"] == -1).mean() > 0.8     # (a few returns share cubes: w >= 2 there)
    # a dense scan with the gate at c = 0.958 (w >= 115): exactly the points
    # below it keep no score and no normal
    mp3 = oracle.Map(_cfg())
    P3 = oracle.PointSet(mp3, oracle.PointsConfig(trig_tsdf=2 * V, c_min=0.958), _tool(), dirs)
    pts, pose = _frame(_wall(), (0.0, 0.0, 0.0), n=6000)
    P3.frame(pts, pose)
    e3 = P3.export()
    w = np.array([mp3.voxel(*x)[1] for x in e3["ijk"]], np.float32)
    low = (w / (w + np.float32(5))) < np.float32(0.958)
    assert 200 < low.sum() < len(low) - 200
    assert (e3["score"][low] == -1).all() and (e3["normal"][low] == 0).all()
    assert (e3["score"][~low] >= 0).mean() > 0.95


def _slotted_scene():
    g = synth.Group(a=np.array([2.02, 0, 0]), b=np.array([2.02, 0, 0]), radius=0.8,
                    boxes=np.array([[2.0, -0.5, -0.5, 2.04, -0.01, 0.5],
                                    [2.0, 0.01, -0.5, 2.04, 0.5, 0.5],
                                    [2.3, -0.5, -0.5, 2.34, 0.5, 0.5]]))
    return synth.Scene([g], *synth._bounds([g]))


def _c2f_expected(mp, tool, dirs, e, ids, snap, stride, half, radius):
    """Brute force of the coarse-to-fine rule from the full per-direction
    score table of the plain scorer: coarse set, centre (nearest other
    point with a direction in `snap`, else the coarse best), window, then the
    lowest-index minimum over the union."""
    G = len(dirs)
    centres = ((e["ijk"][ids].astype(np.float32) + np.float32(0.5)) * np.float32(V))
    _, _, ds = mp.score(tool, dirs, centres, e["normal"][ids], dir_scores=True)
    res_ijk = e["ijk"][snap >= 0].astype(np.int64)
    res_best = snap[snap >= 0]
    out = []
    for k, i in enumerate(ids):
        sc = ds[k]
        d = res_ijk - e["ijk"][i]
        d2 = (d ** 2).sum(1)
        ok = (d2 > 0) & (d2 * float(np.float32(V)) ** 2 <= float(np.float32(radius)) ** 2)
        centre = -1
        if ok.any():
            j = np.lexsort((d[ok, 0], d[ok, 1], d[ok, 2], d2[ok]))[0]
            centre = int(res_best[ok][j])
        coarse = np.arange(0, G, stride)
        if centre < 0:
            cs = [(sc[g], g) for g in coarse if sc[g] >= 0]
            centre = min(cs)[1] if cs else -1
        inE = np.zeros(G, bool)
        inE[coarse] = True
        if centre >= 0:
            dd = np.abs(np.arange(G) - centre)
            inE |= np.minimum(dd, G - dd) <= half
        cand = [(sc[g], g) for g in range(G) if inE[g] and sc[g] >= 0]
        out.append(min(cand) if cand else (tool.n_c + 1, -1))
    return out


def test_coarse_to_fine_search_brute_force():
    """Sec. 3.6's coarse-to-fine search on the paper's yaw ring (D = 180,
    70 degree cone; 20 degree coarse stride, +-24 degree window, 0.3 m)
    against a brute force over the plain scorer's per-direction scores, for
    a first batch (no resolved neighbours: windows around the coarse bests)
    and a second (windows around neighbours' directions). The observation
    filter is disabled so the plain scorer sees the same candidates."""
    dirs = synth.yaw_ring(180)
    tool = _tool(cos_theta_max=synth.COS_70, corr_length=1.0)
    mp = oracle.Map(_cfg())
    pc = oracle.PointsConfig(trig_tsdf=2 * V, budget=0, obs_dot=-2.0, c2f_stride=10, c2f_half=12,
                             c2f_radius=0.3)
    P = oracle.PointSet(mp, pc, tool, dirs)
    pts, pose = _frame(_slotted_scene(), (0.0, 0.0, 0.0), n=6000)
    P.frame(pts, pose)
    before = P.export()
    checked = 0
    for batch in (400, 10 ** 9):
        P.drain(batch)
        after = P.export()
        ids = np.flatnonzero((before["score"] < 0) & (after["score"] >= 0))
        assert len(ids) > 100
        exp = _c2f_expected(mp, tool, dirs, after, ids, before["best"], 10, 12, 0.3)
        got = list(zip(after["score"][ids].tolist(), after["best"][ids].tolist()))
        assert got == [(int(s), int(g)) for s, g in exp]
        checked += len(ids)
        before = after
    assert checked > 1000
    labels = after["label"]
    assert (labels == oracle.ACCESSIBLE).sum() > 50 and (labels == oracle.BLOCKED).sum() > 50
    # a second frame re-queues resolved points: their centre comes from another
    # point (never their own stored direction), and the stored score only
    # decreases (a strictly lower score replaces it, with its direction)
    pts, pose = _frame(_slotted_scene(), (0.0, 0.03, 0.0), n=6000, seed=1)
    P.frame(pts, pose)
    before = P.export()
    P.drain(10 ** 9)
    after = P.export()
    n0 = len(before["score"])
    again = np.flatnonzero((before["score"][:n0] >= 0) & (before["queued"][:n0] == 1))
    assert len(again) > 500
    exp = _c2f_expected(mp, tool, dirs, after, again, before["best"], 10, 12, 0.3)
    for i, (s, g) in zip(again, exp):
        old = (int(before["score"][i]), int(before["best"][i]))
        want = (int(s), int(g)) if s < old[0] else old
        assert (int(after["score"][i]), int(after["best"][i])) == want, i


@pytest.mark.parametrize("stride,half", [(1, 0), (10, 90)])
def test_coarse_to_fine_degenerate_cases_are_the_full_search(stride, half):
    """A stride of 1, or a window of half the ring, searches every direction:
    the same state as the full search."""
    dirs = synth.yaw_ring(180)
    tool = _tool(cos_theta_max=synth.COS_70, corr_length=1.0)
    res = []
    for c2f in (dict(), dict(c2f_stride=stride, c2f_half=half, c2f_radius=0.3)):
        P = oracle.PointSet(oracle.Map(_cfg()), oracle.PointsConfig(trig_tsdf=2 * V, budget=1500,
                                                                    **c2f), tool, dirs)
        for k in range(2):
            pts, pose = _frame(_slotted_scene(), (0.0, 0.05 * k, 0.0), n=4000, seed=k)
            P.frame(pts, pose)
        res.append(P.export())
    for key in ("score", "best", "label", "a"):
        assert (res[0][key] == res[1][key]).all(), key
    assert (res[0]["score"] >= 0).sum() > 1000


_M64 = (1 << 64) - 1


def _mix64(z):
    """splitmix64's output function written out (Steele, Lea, Flood 2014)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def test_mix64_gives_the_published_splitmix64_outputs():
    """The hash that draws the sample: splitmix64 seeded with 0 outputs
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f (the state
    advances by 0x9e3779b97f4a7c15 before each output)."""
    state, out = 0, []
    for _ in range(3):
        state = (state + 0x9E3779B97F4A7C15) & _M64
        out.append(oracle.mix64(state))
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    for z in (0, 1, 2 ** 63, 0x123456789ABCDEF, _M64):
        assert oracle.mix64(z) == _mix64(z)


def _voxel_state(mp):
    e = mp.export()
    return {tuple(map(int, k)): (int(S), int(w), int(c))
            for k, S, w, c in zip(e["ijk"], e["S"], e["w"], e["cleared"])}


def _tsdf(state, k, tau):
    S, w, _ = state.get(tuple(map(int, k)), (0, 0, 0))
    return np.float32(tau) if w == 0 else np.float32(S / (w * 1048576.0))


def _expected_queue(before, after, ijk, frame, sample, radius=3):
    """Sec. 3.5 triggers (i) and (ii) by brute force over the map's voxels:
    the changed voxels (stored state before != after), the sample of the
    `sample` smallest hashes (all if 0), every point within `radius` voxels
    of a sampled one; and the TSDF moving by more than 2v at the point."""
    from scipy.spatial import cKDTree
    changed = np.array([k for k, v in after.items() if before.get(k, (0, 0, 0)) != v], np.int64)
    assert len(changed) > 0
    salt = _mix64(frame)
    h = [_mix64((((x + (1 << 20)) & 0x1FFFFF) | (((y + (1 << 20)) & 0x1FFFFF) << 21) |
                 (((z + (1 << 20)) & 0x1FFFFF) << 42)) ^ salt)
         for x, y, z in changed.tolist()]
    ranked = sorted(range(len(h)), key=lambda i: h[i])
    sel = changed if sample == 0 or len(changed) <= sample else changed[ranked[:sample]]
    d, _ = cKDTree(sel.astype(np.float64)).query(ijk.astype(np.float64),
                                                 distance_upper_bound=radius + 1e-9)
    trig_ii = np.isfinite(d)
    tau = _cfg().tau
    trig_i = np.array([abs(_tsdf(after, k, tau) - _tsdf(before, k, tau)) > np.float32(2 * V)
                       for k in ijk])
    return trig_i, trig_ii, len(changed)


def _two_frames(pc, second, first=None, cfg=None):
    """First frame of the slotted scene, drained; then `second` (points,
    pose) with nothing evaluated. Returns the layer, the voxel states before
    and after the second frame and the count of points before it."""
    mp = oracle.Map(cfg or _cfg())
    P = oracle.PointSet(mp, pc, _tool(), synth.fibonacci_dirs(32))
    pts, pose = first if first is not None else _frame(_slotted_scene(), (0.0, 0.0, 0.0), n=6000)
    P.frame(pts, pose)
    P.drain(10 ** 9)
    n0 = len(P)
    before = _voxel_state(mp)
    P.frame(*second)
    return P, before, _voxel_state(mp), n0


def _side_frame():
    pts, pose = _frame(_slotted_scene(), (0.0, 0.02, 0.0), n=6000, seed=4)
    return pts[pts[:, 1] > 0.2], pose


@pytest.mark.parametrize("sample", [0, 256, 16, 2])
def test_neighbourhood_trigger_against_brute_force(sample):
    """Sec. 3.5 (ii), sampled as the paper samples it: after a second frame
    that sees only part of the scene (the sensor moves 2 cm, below the
    motion trigger), the queued old points are exactly those within r_u = 3v
    of a drawn changed voxel, or whose TSDF moved by more than 2v; new
    points are all queued."""
    P, before, after, n0 = _two_frames(
        oracle.PointsConfig(trig_tsdf=2 * V, budget=0, trig_sample=sample), _side_frame())
    e = P.export()
    trig_i, trig_ii, nchg = _expected_queue(before, after, e["ijk"][:n0], 2, sample)
    queued = e["queued"][:n0].astype(bool)
    assert np.array_equal(queued, trig_i | trig_ii)
    assert e["queued"][n0:].all()
    assert trig_ii.sum() > (100 if sample == 0 or sample > 16 else 10)
    assert (~queued).sum() > 100                          # far points stay unqueued
    if sample:
        assert nchg > sample                                 # the sample is a strict subset


def test_brick_rule_covers_the_neighbourhood_trigger():
    """The brick rule (a touched brick within one brick) queues every point
    that the unsampled voxel rule does, which queues every point the sampled
    rule does; all three leave far points alone."""
    q = {}
    for name, pc in (("brick", dict(trig_exact=0)), ("all", dict(trig_sample=0)),
                     ("sampled", dict(trig_sample=256))):
        P, _, _, n0 = _two_frames(oracle.PointsConfig(trig_tsdf=2 * V, budget=0, **pc),
                                  _side_frame())
        q[name] = P.export()["queued"][:n0].astype(bool)
    assert not (q["all"] & ~q["brick"]).any()
    assert not (q["sampled"] & ~q["all"]).any()
    assert q["brick"].sum() > q["all"].sum() > q["sampled"].sum()
    assert (~q["brick"]).sum() > 100


def test_tsdf_trigger_fires_without_the_neighbourhood_trigger():
    """Sec. 3.5 (i) on its own: the wall moves 6 cm (3 voxels) back and is
    seen by ten times as many returns, so the TSDF at the old surface voxels
    rises from about 0 to about 5 cm, more than 2v; with one changed voxel
    drawn per frame, (ii) misses most of them and (i) alone queues them."""
    wall0 = _wall(x0=2.0, half=0.3)
    wall1 = _wall(x0=2.06, half=0.3)
    first = _frame(wall0, (0.0, 0.0, 0.0), n=2000, seed=1)
    second = _frame(wall1, (0.0, 0.0, 0.0), n=20000, seed=2)
    P, before, after, n0 = _two_frames(
        oracle.PointsConfig(trig_tsdf=2 * V, budget=0, trig_sample=1), second, first=first)
    e = P.export()
    trig_i, trig_ii, _ = _expected_queue(before, after, e["ijk"][:n0], 2, 1)
    assert (trig_i & ~trig_ii).sum() > 50
    assert np.array_equal(e["queued"][:n0].astype(bool), trig_i | trig_ii)


def _pole_and_wall():
    """A wall at x = 2.0 m and, 26 cm in front of it, a 2 x 8 cm pole."""
    boxes = np.array([[2.0, -0.3, -0.3, 2.04, 0.3, 0.3], [1.74, -0.04, -0.3, 1.76, 0.04, 0.3]])
    g = synth.Group(a=np.array([1.9, 0, 0]), b=np.array([1.9, 0, 0]), radius=0.6, boxes=boxes)
    return synth.Scene([g], *synth._bounds([g]))


def test_cleared_band_changes_trigger_on_their_own():
    """A ray-cleared mark is a change of state: the first frame keeps only
    the pole's returns, the second only the wall's. The wall's cleared band,
    stretched to (tau, 4 tau], passes beside the pole and marks voxels there
    that were never touched, while the wall's cubes stay more than r_u away
    from the pole. The pole's points are queued by those marks alone, in the
    brute force and in the oracle; the brick rule reaches them only through
    the bricks of band samples (two bricks from every cube brick)."""
    cfg = _cfg()
    cfg.clear_hi = 4.0
    cfg.clear_samples = 12
    fr1 = _frame(_pole_and_wall(), (0.0, 0.0, 0.0), n=6000, seed=5)
    fr2 = _frame(_pole_and_wall(), (0.0, 0.0, 0.0), n=6000, seed=6)
    first = (fr1[0][fr1[0][:, 0] < 1.9], fr1[1])
    second = (fr2[0][fr2[0][:, 0] > 1.9], fr2[1])
    q = {}
    for name, pc in (("brick", dict(trig_exact=0)), ("all", dict(trig_sample=0))):
        P, before, after, n0 = _two_frames(oracle.PointsConfig(trig_tsdf=2 * V, budget=0, **pc),
                                           second, first=first, cfg=cfg)
        e = P.export()
        q[name] = e["queued"][:n0].astype(bool)
        if name == "all":
            trig_i, trig_ii, _ = _expected_queue(before, after, e["ijk"][:n0], 2, 0)
            assert np.array_equal(q[name], trig_i | trig_ii)
            pole = e["ijk"][:n0, 0] == 87            # every old point is on the pole
            assert pole.all() and not trig_i.any()
            chg_w = [k for k, v in after.items() if before.get(k, (0, 0, 0))[:2] != v[:2]]
            assert min(abs(k[0] - 87) for k in chg_w) > 3   # no S or w change within r_u
            assert trig_ii.sum() > 10
    assert not (q["all"] & ~q["brick"]).any()
