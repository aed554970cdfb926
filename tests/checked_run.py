"""Run by test_gpu_checked.py in a child process with AF_CHECKED=1: the
bounds-checked build (libaf_checked.so) through integration, the bit view,
scoring on the fast and the bounds-checked paths, the stateful point layer
and a batched tick, each compared with the oracle (or the plain path) bit for
bit; every context's device status must stay AF_OK (no check failed)."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle  # noqa: E402
from parity import oracle_config, oracle_tool, to_dev  # noqa: E402
from paper_2608_06412_gb300 import af, synth, workload  # noqa: E402


def main():
    assert os.environ.get("AF_CHECKED") == "1"
    assert b"checked" in af.load(build=False).af_version()
    torch.cuda.set_device(0)
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W, n=8000)
    caps = dict(hash_capacity=1 << 15, pool_blocks=1 << 13, max_returns=1 << 14,
                max_points=1 << 13)
    maps = []
    # the fast path (the scene well inside the box) and the bounds-checked path
    # (a box barely larger than the scene)
    for Wk in (W, workload.Workload(W.name, W.params, W.scene, (9, -4, -5), (8, 8, 10), W.dirs)):
        g = af.Map(Wk.af_config(**caps))
        maps.append(g)
        g.integrate_scan(to_dev(fr.pts), fr.pose)
        g.set_tool(Wk.af_tool(), Wk.dirs)
        sel = slice(0, 600)
        lab, best = g.score(to_dev(pts[sel]), to_dev(nrm[sel]))
        o = oracle.Map(oracle_config(Wk))
        o.integrate(fr.pts, fr.pose)
        gv, ov = af.export_voxels(g.export_blocks()), o.export()
        keep = (ov["w"] > 0) | (ov["cleared"] != 0)
        for k in ("ijk", "S", "w", "cleared", "occ", "known"):
            assert np.array_equal(gv[k].astype(np.int64), ov[k][keep].astype(np.int64)), k
        ol, ob = o.score(oracle_tool(Wk), Wk.dirs, pts[sel], nrm[sel])
        assert np.array_equal(lab.cpu().numpy(), ol) and np.array_equal(best.cpu().numpy(), ob)
    # the stateful point layer over three frames of a moving sensor
    gp = af.Map(W.af_config(**caps))
    maps.append(gp)
    gp.set_tool(W.af_tool(), W.dirs)
    gp.points_enable(af.PointsConfig(trig_tsdf=2 * W.params["v"], budget=300, capacity=1 << 14))
    op = oracle.PointSet(oracle.Map(oracle_config(W)),
                         oracle.PointsConfig(trig_tsdf=2 * W.params["v"], budget=300),
                         oracle_tool(W), W.dirs)
    for k in range(3):
        f2 = synth.cone_frame(W.scene, 4000, 0.01, 700 + k, origin=(0.0, 0.04 * k, 0.0))
        gp.points_frame(to_dev(f2.pts), f2.pose)
        op.frame(f2.pts, f2.pose)
    ge, oe = gp.points_export(), op.export()
    for k in ("ijk", "label", "score", "best", "queued", "nviews"):
        assert np.array_equal(ge[k], oe[k]), k
    # a batched tick of three scenes against the plain path
    S = workload.batch_scenes(3, seed=4, n_lo=500, n_hi=3000)
    bcaps = dict(hash_capacity=1 << 17, pool_blocks=1 << 15, max_returns=1 << 13,
                 max_points=1 << 13)
    mb = [af.Map(Ws.af_config(**bcaps)) for Ws in S]
    mp = [af.Map(Ws.af_config(**bcaps)) for Ws in S]
    maps += mb + mp
    for Ws, a, b in zip(S, mb, mp):
        a.set_tool(Ws.af_tool(), Ws.dirs)
        b.set_tool(Ws.af_tool(), Ws.dirs)
    batch = af.Batch(mb)
    for f in range(2):
        items = []
        for Ws in S:
            fr2, p2, n2 = workload.pine_frame(Ws, f)
            items.append((to_dev(fr2.pts), fr2.pose, to_dev(p2), to_dev(n2),
                          torch.empty(len(p2), dtype=torch.uint8, device="cuda"),
                          torch.empty(len(p2), dtype=torch.int16, device="cuda")))
        batch.tick(items)
        for it, m in zip(items, mp):
            m.integrate_scan(it[0], it[1])
            lab, best = m.score(it[2], it[3])
            torch.cuda.synchronize()
            assert torch.equal(lab, it[4]) and torch.equal(best, it[5])
    batch.close()
    status = [m.sync_status() for m in maps]
    assert all(s == 0 for s in status), status
    print("CHECKED OK")


if __name__ == "__main__":
    main()
