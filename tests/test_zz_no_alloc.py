"""af_integrate_scan_noalloc, the entry point for callers that cannot
allocate device memory (a real-time loop with memory fixed at start-up, a
framework that owns all device buffers): integrating into a caller-owned
dense voxel box must give exactly what the allocating map path
(af_create + af_integrate_scan) gives for the same voxels, call after call.

This file is collected last on purpose; it must pass on its own in a fresh
process as well as after the rest of the suite."""
import numpy as np
import pytest

from paper_2608_06412_gb300 import af, workload

pytestmark = pytest.mark.gpu


def _densify(blocks, box_min, box_dim):
    """The map path's exported bricks as the dense box layout."""
    bx, by, bz = (int(d) for d in box_dim)
    vox = np.zeros(bx * by * bz, np.uint64)
    flags = np.zeros(bx * by * bz, np.uint8)
    l = np.arange(512)
    loc = np.stack([l & 7, (l >> 3) & 7, l >> 6], 1)
    ijk = (blocks["key"][:, None, :] * 8 + loc[None]).reshape(-1, 3) - np.asarray(box_min)
    inside = ((ijk >= 0) & (ijk < np.asarray(box_dim))).all(1)
    at = (ijk[:, 2] * by + ijk[:, 1]) * bx + ijk[:, 0]
    S = blocks["S"].reshape(-1)
    w = blocks["w"].reshape(-1)
    vox[at[inside]] = ((S[inside].astype(np.int64) << 20) |
                       w[inside].astype(np.int64)).view(np.uint64)
    flags[at[inside]] = blocks["flags"].reshape(-1)[inside]
    return vox, flags


@pytest.mark.parametrize("sub_box,clamp_signed", [(False, 0), (True, 0), (True, 1)])
def test_noalloc_matches_map_path_on_consecutive_scans(sub_box, clamp_signed):
    import torch
    W = workload.single_frame()
    fr, _, _ = workload.single_frame_inputs(W)
    cfg = W.af_config(clamp_signed=clamp_signed, w_cap=3 if clamp_signed else 2000)
    # scan A in the world frame; scan B seen from a rotated, shifted sensor
    a = fr.pts[:10000]
    R = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    t = np.array([0.1, -0.05, 0.02])
    pose_b = np.eye(4)
    pose_b[:3, :3], pose_b[:3, 3] = R, t
    b = ((fr.pts[10000:].astype(np.float64) - t) @ R).astype(np.float32)
    scans = [(a, fr.pose), (b, pose_b.astype(np.float32))]

    dom_min = np.array(W.dom_min) * 8
    dom_dim = np.array(W.dom_bricks) * 8
    if sub_box:   # a box that cuts through the scene
        box_min = dom_min + dom_dim // 3
        box_dim = dom_dim // 2
    else:
        box_min, box_dim = dom_min, dom_dim
    count = int(np.prod(box_dim))

    g = af.Map(cfg)
    vox = torch.zeros(count, dtype=torch.int64, device="cuda")
    flags = torch.zeros(count, dtype=torch.uint8, device="cuda")
    for xyz, pose in scans:
        d = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
        g.integrate_scan(d, pose)
        af.integrate_scan_noalloc(cfg, d, pose, box_min, box_dim, vox, flags)
        torch.cuda.synchronize()
        ref_vox, ref_flags = _densify(g.export_blocks(), box_min, box_dim)
        got_vox = vox.cpu().numpy().view(np.uint64)
        got_flags = flags.cpu().numpy()
        assert (ref_vox != 0).sum() > 1000
        np.testing.assert_array_equal(got_vox, ref_vox)
        np.testing.assert_array_equal(got_flags, ref_flags)


@pytest.mark.parametrize("clamp_signed", [0, 1])
def test_noalloc_matches_oracle_on_consecutive_scans(clamp_signed):
    """Every voxel of a box that cuts through the scene, after each of two
    scans (the second from a rotated, shifted sensor), against the oracle
    (Sec. 3.2, 3.4): S, w, the ray-cleared mark and the occupied / known rule,
    bit for bit."""
    import torch
    import oracle
    from parity import oracle_config
    W = workload.single_frame()
    fr, _, _ = workload.single_frame_inputs(W)
    cfg = W.af_config(clamp_signed=clamp_signed, w_cap=3 if clamp_signed else 2000)
    om = oracle.Map(oracle_config(W, clamp_signed=clamp_signed,
                                  w_cap=3 if clamp_signed else 2000))
    a = fr.pts[:10000]
    R = np.array([[0.0, 0, 1], [0, 1, 0], [-1, 0, 0]])
    t = np.array([-0.08, 0.03, 0.05])
    pose_b = np.eye(4)
    pose_b[:3, :3], pose_b[:3, 3] = R, t
    b = ((fr.pts[10000:].astype(np.float64) - t) @ R).astype(np.float32)
    scans = [(a, np.asarray(fr.pose, np.float32)), (b, pose_b.astype(np.float32))]

    # the scene's voxels span x 66..134, y and z -29..28: a box that cuts it on
    # every axis, so that contributions fall both inside and outside
    box_min = np.array([100, -10, -40])
    box_dim = np.array([30, 50, 45])
    count = int(np.prod(box_dim))
    vox = torch.zeros(count, dtype=torch.int64, device="cuda")
    flags = torch.zeros(count, dtype=torch.uint8, device="cuda")
    for xyz, pose in scans:
        om.integrate(xyz, pose)
        d = torch.from_numpy(np.ascontiguousarray(xyz)).cuda()
        af.integrate_scan_noalloc(cfg, d, pose, box_min, box_dim, vox, flags)
        torch.cuda.synchronize()
        e = om.export()
        rel = e["ijk"] - box_min
        inside = ((rel >= 0) & (rel < box_dim)).all(1)
        at = (rel[inside, 2] * box_dim[1] + rel[inside, 1]) * box_dim[0] + rel[inside, 0]
        ref_vox = np.zeros(count, np.int64)
        ref_flags = np.zeros(count, np.uint8)
        ref_vox[at] = (e["S"][inside].astype(np.int64) << 20) | e["w"][inside].astype(np.int64)
        ref_flags[at] = (e["cleared"][inside] | (e["occ"][inside] << 1) |
                         (e["known"][inside] << 2)).astype(np.uint8)
        got_vox = vox.cpu().numpy()
        got_flags = flags.cpu().numpy()
        assert (ref_vox != 0).sum() > 1000 and (ref_flags & 1).sum() > 100
        assert (~inside).sum() > 1000
        bad = np.nonzero(got_vox != ref_vox)[0]
        assert len(bad) == 0, f"{len(bad)} voxel words differ, first at {bad[0]}"
        np.testing.assert_array_equal(got_flags, ref_flags)


def test_noalloc_rejects_scans_beyond_its_fixed_scratch():
    import torch
    W = workload.single_frame()
    cfg = W.af_config()
    n = af.NOALLOC_MAX_RETURNS + 1
    xyz = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    vox = torch.zeros(8, dtype=torch.int64, device="cuda")
    flags = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(af.AfError) as e:
        af.integrate_scan_noalloc(cfg, xyz, np.eye(4), np.zeros(3), (2, 2, 2), vox, flags)
    assert e.value.status == af.ERR_CAPACITY
    assert "scratch" in str(e.value)
