"""Parity at the large-map size: 8 pines on a noisy 40 x 40 m ground, 3,000
frames of 20k returns (375 orbit frames around each pine), v = 1 cm,
tau = 4 cm (9^3 cube), K = 256 (G = 512), corridor 1.5 m. The GPU
integrates the whole stream and scores every surface point of it (one per
voxel hit); sampled voxel clusters and point clusters are checked bit for
bit against an oracle built from only the returns that can affect them: a
voxel's state depends on returns whose cube holds it or whose cleared band
reaches it (within 0.15 m), a point's label on voxels within its kernels'
reach (L + L_c + r = 1.8 m), so on returns within 2.0 m. The soft clearance
and its refinement run on the brick-sparse SDF view (the box's dense view
would need over 2^31 cells) and are checked against the oracle on a sampled
point cluster."""
import numpy as np
import pytest

import oracle
from parity import oracle_config, oracle_tool, to_dev
from paper_2608_06412_gb300 import af, workload

pytestmark = pytest.mark.gpu

VOXEL_RADIUS = 0.15
POINT_RADIUS = 2.0
CAPS = dict(hash_capacity=1 << 23, pool_blocks=1 << 22, max_returns=1 << 15,
            max_points=1 << 20)


@pytest.fixture(scope="module")
def large():
    import torch
    W = workload.large_map()
    frames = workload.large_frames(W, range(W.params["frames"]))
    g = af.Map(W.af_config(**CAPS))
    g.set_tool(W.af_tool(), W.dirs)
    for pts, pose, _, _, _ in frames:
        g.integrate_scan(to_dev(pts), pose)
    torch.cuda.synchronize()
    assert g.sync_status() == 0
    # every surface point of the stream, one per voxel (first occurrence)
    P = np.concatenate([f[3] for f in frames])
    N = np.concatenate([f[4] for f in frames])
    v = np.float64(np.float32(W.params["v"]))
    ijk = np.floor(P.astype(np.float64) / v).astype(np.int64) + (1 << 20)
    key = ijk[:, 0] | (ijk[:, 1] << 21) | (ijk[:, 2] << 42)
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)
    P, N = np.ascontiguousarray(P[first]), np.ascontiguousarray(N[first])
    lab = np.empty(len(P), np.uint8)
    best = np.empty(len(P), np.int16)
    chunk = CAPS["max_points"]
    for a in range(0, len(P), chunk):
        l, b = g.score(to_dev(P[a:a + chunk]), to_dev(N[a:a + chunk]))
        lab[a:a + chunk] = l.cpu().numpy()
        best[a:a + chunk] = b.cpu().numpy()
    assert g.sync_status() == 0
    return W, frames, g, P, N, lab, best


def _oracle_near(W, frames, centres, radius):
    """Oracle map from every return within `radius` of a centre, scan by
    scan in stream order."""
    from scipy.spatial import cKDTree
    centres = np.asarray(centres, np.float64)
    lo, hi = centres.min(0) - radius, centres.max(0) + radius
    tree = cKDTree(centres)
    om = oracle.Map(oracle_config(W))
    for pts, pose, world, _, _ in frames:
        box = np.all((world >= lo) & (world <= hi), axis=1)
        if not box.any():
            continue
        idx = np.nonzero(box)[0]
        d, _ = tree.query(world[idx].astype(np.float64), distance_upper_bound=radius)
        sel = idx[np.isfinite(d)]
        if len(sel):
            om.integrate(pts[sel], pose)
    return om


def test_large_map_scale(large):
    W, frames, g, P, N, lab, best = large
    st = g.stats()
    assert st["scans"] == W.params["frames"]
    assert len(P) > 2_000_000, len(P)
    assert st["blocks_allocated"] > 100_000
    assert (lab == af.ACCESSIBLE).any() and (lab == af.BLOCKED).any()


@pytest.mark.parametrize("which", [0, 1])
def test_sampled_voxels_bit_exact(large, which):
    W, frames, g, P, N, lab, best = large
    gv = af.export_voxels(g.export_blocks(cap=40_000))
    rng = np.random.default_rng(40 + which)
    seed = rng.choice(np.nonzero(gv["w"] > 0)[0])
    near = np.nonzero(np.abs(gv["ijk"] - gv["ijk"][seed]).max(1) <= 6)[0]
    sel = rng.choice(near, min(60, len(near)), replace=False)
    v = np.float64(np.float32(W.params["v"]))
    om = _oracle_near(W, frames, (gv["ijk"][sel] + 0.5) * v, VOXEL_RADIUS)
    for k in sel:
        i, j, l = (int(x) for x in gv["ijk"][k])
        S, w, cl = om.voxel(i, j, l)
        assert (int(gv["S"][k]), int(gv["w"][k]), int(gv["cleared"][k])) == (S, w, cl), (i, j, l)
        assert int(gv["occ"][k]) == om.occ(i, j, l) and int(gv["known"][k]) == om.known(i, j, l)


def test_sampled_points_labels(large):
    """Accessible and blocked points around one accessible point, scored
    against one oracle map built for all of them."""
    W, frames, g, P, N, lab, best = large
    rng = np.random.default_rng(8)
    acc, blk = lab == af.ACCESSIBLE, lab == af.BLOCKED
    # an accessible seed with blocked points nearby
    for seed in rng.permutation(np.nonzero(acc)[0])[:2000]:
        d = np.linalg.norm(P - P[seed], axis=1)
        if (blk & (d < 0.3)).sum() >= 6:
            break
    d = np.linalg.norm(P - P[seed], axis=1)
    near = np.concatenate([np.nonzero(acc & (d < 0.3))[0][:8], np.nonzero(blk & (d < 0.3))[0][:8]])
    om = _oracle_near(W, frames, P[near].astype(np.float64), POINT_RADIUS)
    ol, ob = om.score(oracle_tool(W), W.dirs, P[near], N[near])
    np.testing.assert_array_equal(lab[near], ol)
    np.testing.assert_array_equal(best[near], ob)
    assert (ol == af.ACCESSIBLE).sum() >= 4 and (ol == af.BLOCKED).sum() >= 4


def test_sampled_soft_refinement_sparse_view(large):
    """The differentiable step on the large map: the dense view does not fit
    the 40 x 40 m box at 1 cm, so the brick-sparse one is built; C before and
    after 20 ascent steps from the best table direction of a cluster of
    accessible points, within 1e-5 m of the oracle's trajectories."""
    import torch
    W, frames, g, P, N, lab, best = large
    M = W.af_config(**CAPS)
    cells = 1
    for k in range(3):
        cells *= 8 * M.domain_bricks[k] + 1
    assert cells >= 1 << 31                      # automatic choice: the sparse view
    rng = np.random.default_rng(13)
    acc = np.nonzero(lab == af.ACCESSIBLE)[0]
    seed = rng.choice(acc)
    near = acc[np.argsort(np.linalg.norm(P[acc] - P[seed], axis=1))[:24]]
    Pd, Nd = to_dev(P[near]), to_dev(N[near])
    l, b = g.score(Pd, Nd)
    u0 = g.soft_start(l, b)
    z = torch.zeros(len(near), dtype=torch.float32, device="cuda")
    c0 = g.soft_clearance_raw(Pd, u0, z, z, z, 1).cpu().numpy()
    al, be, hh = z.clone(), z.clone(), z.clone()
    c, cmin = g.soft_refine(Pd, u0, al, be, hh, 1, steps=20, lr_dir=0.05, lr_h=0.005, h_max=0.05)
    c, cmin, hh = c.cpu().numpy(), cmin.cpu().numpy(), hh.cpu().numpy()
    assert g.sync_status() == 0
    om = _oracle_near(W, frames, P[near].astype(np.float64), POINT_RADIUS + 0.05)
    tool = oracle_tool(W)
    pts, dirs0 = P[near], W.dirs[best[near]]
    zz = np.zeros(len(near), np.float32)
    oc0, _ = om.soft_clearance(tool, pts, 1, dirs0, zz, zz, zz, af.TAU_S)
    np.testing.assert_allclose(c0, oc0, rtol=0, atol=1e-5)
    ra, rb, rh, rc, rm = om.soft_refine(tool, pts, 1, dirs0, zz, zz, zz, 20, 0.05, 0.005, 0.05)
    close = np.abs(c - rc) <= 1e-5
    # a trajectory may part from the oracle's at a kink met within rounding
    assert close.sum() >= len(close) - 1, np.abs(c - rc)
    assert (np.abs(cmin - rm)[close] <= 1e-5).all()
    assert (np.abs(hh - rh)[close] <= 1e-4).all()
    assert np.ptp(c0) > 0                        # the samples read the map, not only tau
