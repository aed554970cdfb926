"""Pins of the oracle's accessibility scoring against what the paper fixes.

Kernels (Sec. 3.4): hand counts for an axis-aligned direction
(tests/golden/kernel_axis.txt) and a box-versus-cylinder geometric check for
tilted directions. Scoring (Sec. 3.4, 3.5, 4.1): hand-built single-direction
scenes for every term of the score, the lowest-index tie-break, the
confidence gate, and the paper's qualitative ground truth on exactly
voxelised analytic scenes -- a slot narrower than the tool is inaccessible,
a convex sphere and a flat wall are accessible near their normals (Tab. 1),
and adding geometry never turns a blocked point accessible. Scoring with
kernel tables built once equals scoring that builds them per call. Parity
status: pinned.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import golden
from paper_2608_06412_gb300 import synth

Q = 2.0 ** 20


def _triples(s):
    return [tuple(int(x) for x in part.split()) for part in s.split(";")]


def _tool(**kw):
    base = dict(radius=0.04, length=0.25, self_excl=0.04, corr_radius=0.05,
                corr_length=1.0, cos_theta_max=0.0, n_c=5, strict=0)
    base.update(kw)
    return oracle.Tool(**base)


def _cfg(v=0.02, tau=0.06, dom=((-512,) * 3, (1024,) * 3), **kw):
    return oracle.Config(v=v, tau=tau, r_c=v / 2, cube_radius=3, clear_samples=8,
                         dom_min=dom[0], dom_size=dom[1], **kw)


def _voxelise(mp, sdf, lo, hi, v, tau, band):
    """The paper's ground-truth setting (Sec. 4.1) on the voxel grid: every
    voxel of the box [lo, hi] whose centre's exact signed distance is below
    `band` gets w = 10 observations of clamp(sdf, 0, tau)."""
    ax = [np.arange(lo[k], hi[k] + 1) for k in range(3)]
    ijk = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    c = (ijk + 0.5) * np.float64(np.float32(v))
    d = sdf(c)
    keep = d < band
    dq = np.rint(np.clip(d[keep], 0.0, tau) * Q).astype(np.uint64)
    mp.set_voxels(ijk[keep], dq * np.uint64(10), 10)
    return ijk, d


# ----------------------------------------------------------------------------
# Kernels
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [(0, 0, 1), (1, 0, 0), (0, -1, 0)])
def test_kernel_axis_hand_count(axis):
    g = golden("kernel_axis.txt")
    t = _tool(radius=float(g["tool_radius"]), length=float(g["tool_length"]),
              self_excl=float(g["self_excl"]), corr_radius=float(g["corr_radius"]),
              corr_length=float(g["corr_length"]))
    v = float(g["v"])
    tool = oracle.kernel_offsets(t, v, axis, oracle.KERNEL_TOOL)
    corr = oracle.kernel_offsets(t, v, axis, oracle.KERNEL_CORRIDOR)
    assert len(tool) == int(g["tool_count"])
    assert len(corr) == int(g["corridor_count"])
    a = np.abs(np.array(axis))
    layer = (corr @ a.astype(np.int32)) * int(np.sum(axis))
    # every corridor layer holds the same disc of 21 offsets
    _, counts = np.unique(layer, return_counts=True)
    assert set(counts.tolist()) == {int(g["corridor_layer_count"])}
    # the tool rests on the tip: no offset behind it
    assert ((tool @ np.array(axis)) >= 0).all()
    arm = oracle.arm_offsets(v, float(g["tau"]), axis)
    expect = np.array(_triples(g["arm"]))
    perm = {(0, 0, 1): [0, 1, 2], (1, 0, 0): [2, 0, 1], (0, -1, 0): [0, 2, 1]}[axis]
    sign = np.array(axis)[np.argmax(np.abs(axis))]
    np.testing.assert_array_equal(arm, expect[:, perm] * sign if sign < 0 else expect[:, perm])


def _box_vs_cylinder(o, v, u, a0, a1, r, rs_excl=None):
    """Geometric classification of voxel boxes against the finite cylinder
    {a in [a0, a1], |e - a u| <= r} (minus the ball |e| <= rs_excl): +1 when
    the whole box is inside, -1 when the box misses it, 0 when it straddles."""
    h = v / 2
    corners = np.array([[sx, sy, sz] for sx in (-h, h) for sy in (-h, h) for sz in (-h, h)])
    c = o * v
    pts = c[:, None, :] + corners[None]
    a = pts @ u
    rad = np.linalg.norm(pts - a[..., None] * u, axis=-1)
    inside = ((a >= a0) & (a <= a1) & (rad <= r)).all(1)
    half = v * math.sqrt(3) / 2
    ac = c @ u
    rc = np.linalg.norm(c - ac[:, None] * u, axis=1)
    miss = (ac < a0 - half) | (ac > a1 + half) | (rc > r + half)
    if rs_excl is not None:
        far = np.linalg.norm(pts, axis=-1).min(1) > rs_excl
        near = np.linalg.norm(pts, axis=-1).max(1) <= rs_excl
        inside &= far
        miss |= near
    return np.where(inside, 1, np.where(miss, -1, 0))


@pytest.mark.parametrize("gi", [3, 17, 40, 63])
def test_kernel_matches_box_cylinder_geometry(gi):
    """Tilted directions: voxels whose box lies inside the tool / corridor
    cylinder are in the kernel, voxels whose box misses it are not."""
    v = 0.02
    t = _tool()
    u32 = synth.fibonacci_dirs(64)[gi]
    u = u32.astype(np.float64)
    B = 70
    ax = np.arange(-B, B + 1)
    o = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    for which, a0, a1, r, rs in ((oracle.KERNEL_TOOL, 0.0, 0.25, 0.04, 0.04),
                                 (oracle.KERNEL_CORRIDOR, 0.25, 1.25, 0.05, None)):
        k = oracle.kernel_offsets(t, v, u32, which)
        ks = set(map(tuple, k.tolist()))
        cls = _box_vs_cylinder(o, v, u, a0, a1, r, rs)
        ins = [tuple(x) for x in o[cls == 1].tolist()]
        out = [tuple(x) for x in o[cls == -1].tolist()]
        assert all(x in ks for x in ins)
        assert not any(x in ks for x in out)
        assert len(ins) > 0.25 * len(ks)


# ----------------------------------------------------------------------------
# Score composition on hand-built scenes (one direction, u = +z)
# ----------------------------------------------------------------------------

def _one_dir_map(occupied=(), unknown=(), strict=0):
    """Point at voxel (0,0,0) (w = 10, far from any surface); every voxel of
    the +z column region is known-free except `unknown`; `occupied` voxels
    read TSDF = 0."""
    mp = oracle.Map(_cfg())
    ax = np.arange(-4, 5)
    az = np.arange(-2, 70)
    ijk = np.stack(np.meshgrid(ax, ax, az, indexing="ij"), -1).reshape(-1, 3)
    keep = np.array([tuple(x) not in set(unknown) for x in ijk.tolist()])
    mp.set_voxels(ijk[keep], 0, 0, 1)                       # known-free (ray-cleared)
    mp.set_voxel(0, 0, 0, int(0.06 * Q) * 10, 10)            # the scored point
    for o in occupied:
        mp.set_voxel(*o, 0, 10)
    return mp


def _score_one(mp, strict=0):
    s = np.array([[0.01, 0.01, 0.01]], np.float32)
    n = np.array([[0, 0, 1]], np.float32)
    d = np.array([[0, 0, 1]], np.float32)
    lab, best, ds = mp.score(_tool(strict=strict), d, s, n, dir_scores=True)
    return int(lab[0]), int(best[0]), int(ds[0, 0])


@pytest.mark.parametrize("occupied,score,label", [
    ((), 0, oracle.ACCESSIBLE),
    (((0, 0, 5), (1, 0, 6), (0, -1, 9)), 3, oracle.ACCESSIBLE),      # 3 tool hits
    (((0, 0, 5), (1, 0, 6), (0, -1, 9), (2, 0, 10), (0, 0, 12)), 5, oracle.BLOCKED),
    (tuple((0, 0, k) for k in (3, 5, 6, 8, 9, 10, 11)), 5, oracle.BLOCKED),  # saturates at n_c
    (((3, 0, 5), (2, 1, 8), (0, 0, -1), (0, 0, 13 + 50)), 0, oracle.ACCESSIBLE),  # all outside
    (((0, 0, 1), (1, 1, 1), (0, 1, 0)), 0, oracle.ACCESSIBLE),        # self-excluded
    (((0, 0, 30),), 6, oracle.BLOCKED),                               # corridor hit
    (((0, 2, 62),), 6, oracle.BLOCKED),                               # corridor rim, last layer
])
def test_score_terms_hand_built(occupied, score, label):
    """Sec. 3.4: collision count over the tool kernel minus the self-exclusion
    ball, saturating at n_c; any occupied corridor voxel blocks (n_c + 1);
    ACCESSIBLE iff the best score is below n_c."""
    assert _score_one(_one_dir_map(occupied)) == (label, 0, score)


def test_arm_samples_block_unknown_and_occupied():
    """Sec. 3.4: arm-path samples at {0.6, 1.25, 2.25} tau block when occupied
    or unknown (w = 0 and not ray-cleared); other unknown voxels read free."""
    assert _score_one(_one_dir_map(unknown=[(0, 0, 7)])) == (oracle.BLOCKED, 0, 6)
    assert _score_one(_one_dir_map(unknown=[(0, 0, 2)])) == (oracle.BLOCKED, 0, 6)
    assert _score_one(_one_dir_map(occupied=[(0, 0, 4)])) == (oracle.BLOCKED, 0, 6)
    # an unknown voxel off the arm samples, in the tool and in the corridor
    assert _score_one(_one_dir_map(unknown=[(0, 0, 6), (0, 0, 30)])) == (oracle.ACCESSIBLE, 0, 0)
    # ... unless unknown corridor voxels are declared blocking
    assert _score_one(_one_dir_map(unknown=[(0, 0, 30)]), strict=1) == (oracle.BLOCKED, 0, 6)


def test_best_is_lowest_index_minimum_and_gates():
    mp = _one_dir_map(occupied=[(0, 0, 5), (0, 1, 6)])        # +z scores 2
    s = np.array([[0.01, 0.01, 0.01]] * 4, np.float32)
    dirs = np.array([[0, 0, 1], [0, 0, -1], [0, 0, 1], [0, 1, 0]], np.float32)
    n = np.array([[0, 0, 1], [0, 0, 1], [0, 0, 0], [0, 0, 1]], np.float32)
    lab, best, ds = mp.score(_tool(), dirs, s, n, dir_scores=True)
    # point 0: candidates 0 and 2 (both +z, score 2): the lower index wins
    assert (lab[0], best[0]) == (oracle.ACCESSIBLE, 0)
    assert ds[0].tolist() == [2, -1, 2, -1]
    # zero normal: no candidate at all -> BLOCKED with no direction
    assert (lab[2], best[2]) == (oracle.BLOCKED, -1)
    # a point whose voxel is below the confidence gate is not scored (Sec. 3.5)
    lab2, best2 = mp.score(_tool(), dirs, np.array([[0.11, 0.01, 0.01]], np.float32),
                           n[:1])
    assert (lab2[0], best2[0]) == (oracle.UNSCORED, -1)
    mp.set_voxel(5, 0, 0, 0, 2)
    assert mp.score(_tool(), dirs, np.array([[0.11, 0.01, 0.01]], np.float32), n[:1])[0][0] \
        == oracle.UNSCORED
    mp.set_voxel(5, 0, 0, 0, 3)
    assert mp.score(_tool(), dirs, np.array([[0.11, 0.01, 0.01]], np.float32), n[:1])[0][0] \
        != oracle.UNSCORED


# ----------------------------------------------------------------------------
# Paper-level ground truth on exactly voxelised analytic scenes (Sec. 4.1)
# ----------------------------------------------------------------------------

def _slot_scene(half_width):
    """Plate x in [0, 4) cm, |y|, |z| <= 40 cm, with a slot |y| < half_width;
    a solid target slab x >= 10 cm behind it (seen from -x)."""
    v, tau = 0.02, 0.06
    mp = oracle.Map(_cfg())

    def sdf(c):
        plate = np.maximum.reduce([-c[:, 0], c[:, 0] - 0.04, np.abs(c[:, 1]) - 0.4,
                                   np.abs(c[:, 2]) - 0.4])
        slot = half_width - np.abs(c[:, 1])
        plate = np.maximum(plate, np.minimum(slot, 0.4))
        slab = 0.10 - c[:, 0]
        return np.minimum(plate, slab)

    _voxelise(mp, sdf, (-70, -40, -40), (40, 40, 40), v, tau, band=10.0)
    return mp


def test_slot_narrower_than_tool_is_inaccessible():
    """A 3 cm slot is narrower than the 8 cm tool: target points behind it are
    BLOCKED for every candidate; a 24 cm slot lets the tool through along -x."""
    dirs = np.concatenate([[[-1, 0, 0]], synth.fibonacci_dirs(64)]).astype(np.float32)
    pts = np.array([[0.11, y, z] for y in (-0.01, 0.01) for z in (-0.05, 0.01, 0.07)],
                   np.float32)
    nrm = np.tile(np.array([[-1, 0, 0]], np.float32), (len(pts), 1))
    lab, best = _slot_scene(0.015).score(_tool(), dirs, pts, nrm)
    assert (lab == oracle.BLOCKED).all()
    lab, best, ds = _slot_scene(0.12).score(_tool(), dirs, pts, nrm, dir_scores=True)
    assert (lab == oracle.ACCESSIBLE).all() and (best == 0).all()


def test_convex_sphere_accessible_near_normal():
    """Sphere (Tab. 1: F1 = 100, no false negatives): every scored surface
    point is ACCESSIBLE, and the candidate closest to its normal is an
    accessible direction (score below n_c)."""
    v, tau, R = 0.02, 0.06, 0.3
    mp = oracle.Map(_cfg())
    ijk, d = _voxelise(mp, lambda c: np.linalg.norm(c, axis=1) - R,
                       (-45, -45, -45), (44, 44, 44), v, tau, band=0.2)
    surf = ijk[np.abs(d) < v / 2]
    rng = np.random.default_rng(0)
    surf = surf[rng.choice(len(surf), 150, replace=False)]
    pts = ((surf + 0.5) * np.float32(v)).astype(np.float32)
    nrm = (pts / np.linalg.norm(pts, axis=1, keepdims=True)).astype(np.float32)
    dirs = synth.fibonacci_dirs(64)
    lab, best, ds = mp.score(_tool(), dirs, pts, nrm, dir_scores=True)
    assert (lab == oracle.ACCESSIBLE).all()
    nearest = np.argmax(nrm @ dirs.T, axis=1)
    assert (ds[np.arange(len(pts)), nearest] < 5).all()     # an accessible direction
    spacing = math.sqrt(4 * math.pi / 64)
    ang = np.arccos(np.clip(np.sum(nrm * dirs[best], 1), -1, 1))
    assert (ang < math.pi / 2).all() and np.median(ang) < 3 * spacing


def test_flat_wall_accessible_along_normal():
    """Wall (Tab. 1: F1 = 100): every point of a flat wall is ACCESSIBLE and
    the direction along its normal scores 0."""
    v, tau = 0.02, 0.06
    mp = oracle.Map(_cfg())
    _voxelise(mp, lambda c: -c[:, 0], (-70, -30, -30), (10, 30, 30), v, tau, band=10.0)
    dirs = np.concatenate([[[-1, 0, 0]], synth.fibonacci_dirs(64)]).astype(np.float32)
    pts = np.array([[0.01, y, z] for y in np.arange(-0.19, 0.2, 0.06)
                    for z in np.arange(-0.19, 0.2, 0.06)], np.float32)
    nrm = np.tile(np.array([[-1, 0, 0]], np.float32), (len(pts), 1))
    lab, best, ds = mp.score(_tool(), dirs, pts, nrm, dir_scores=True)
    assert (lab == oracle.ACCESSIBLE).all() and (best == 0).all()
    assert (ds[:, 0] == 0).all()


def test_adding_geometry_never_unblocks():
    """Occupancy grows (occ' contains occ): every direction score is >= and no
    label moves from BLOCKED to ACCESSIBLE (the monotonicity the method
    relies on)."""
    rng = np.random.default_rng(42)
    v = 0.02
    t = _tool(length=0.1, corr_length=0.2)
    mp = oracle.Map(_cfg())
    lo, hi = -14, 14
    ax = np.arange(lo, hi + 1)
    ijk = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    r = rng.uniform(size=len(ijk))
    occ = r < 0.004
    known = r < 0.95
    mp.set_voxels(ijk[known & ~occ], np.uint64(int(0.05 * Q) * 10), 10)
    mp.set_voxels(ijk[occ], 0, 10)
    pidx = rng.integers(-6, 7, size=(60, 3))
    mp.set_voxels(pidx, np.uint64(int(0.05 * Q) * 10), 10)
    pts = ((pidx + 0.5) * np.float32(v)).astype(np.float32)
    nrm = rng.normal(size=(60, 3)).astype(np.float32)
    dirs = synth.fibonacci_dirs(32)
    lab0, _, ds0 = mp.score(t, dirs, pts, nrm, dir_scores=True)
    add = ijk[(rng.uniform(size=len(ijk)) < 0.004)]
    mp.set_voxels(add, 0, 10)
    lab1, _, ds1 = mp.score(t, dirs, pts, nrm, dir_scores=True)
    cand = ds0 >= 0
    assert (ds1[cand] >= ds0[cand]).all()
    assert not ((lab0 == oracle.BLOCKED) & (lab1 == oracle.ACCESSIBLE)).any()
    assert (ds1[cand] > ds0[cand]).any()       # the added geometry mattered
    assert (lab0 == oracle.ACCESSIBLE).any()


def test_prebuilt_tables_score_identically():
    """or_score_tables with kernel tables built once gives exactly what
    or_score (which builds them per call) gives, on two maps in turn."""
    from paper_2608_06412_gb300 import workload
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W, n=4000)
    p = W.map_params()
    cfg = oracle.Config(v=p["v"], tau=p["tau"], r_c=p["r_c"], cube_radius=p["cube_radius"],
                        clear_samples=p["clear_samples"], dom_min=tuple(8 * b for b in W.dom_min),
                        dom_size=tuple(8 * b for b in W.dom_bricks), w_min=p["w_min"])
    tool = oracle.Tool(**W.tool())
    T = oracle.ScoreTables(cfg, tool, W.dirs)
    sel = slice(0, 400)
    for half in (fr.pts[:2000], fr.pts):
        mp = oracle.Map(cfg)
        mp.integrate(half, fr.pose)
        a = mp.score(tool, W.dirs, pts[sel], nrm[sel], dir_scores=True)
        b = mp.score_tables(T, pts[sel], nrm[sel], dir_scores=True)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert (a[0] == oracle.ACCESSIBLE).any() and (a[0] == oracle.BLOCKED).any()
    with pytest.raises(ValueError):
        oracle.Map(oracle.Config(v=0.01, tau=0.04, r_c=0.005, cube_radius=4, clear_samples=10,
                                 dom_min=(0, 0, 0), dom_size=(8, 8, 8))).score_tables(T, pts[:1],
                                                                                       nrm[:1])
