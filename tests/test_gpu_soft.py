"""The differentiable form on the GPU (af_soft_*), against the FP64 oracle on
the same seeded inputs: seeds bit-exact; C and the hard clearance within
1e-5 m; the adjoint within 1e-3 of the oracle's gradient; the adjoint against
central finite differences of the GPU's own single-precision C (h = 1e-4) on
every pair where the oracle shows the difference interval free of the kinks
of trilinear interpolation, per pair within 1e-3 relative plus what single
precision lets the difference resolve (measured against the oracle); the autograd Function equal to the adjoint;
refinement and the per-point best exactly self-consistent and within
tolerance of the oracle's trajectories; views rebuilt after a new scan; the
brick-sparse view giving the dense view's results bit for bit."""
import numpy as np
import pytest

import oracle
from parity import oracle_config, oracle_tool, to_dev
from paper_2608_06412_gb300 import af, synth, workload

pytestmark = pytest.mark.gpu

CAPS = dict(hash_capacity=1 << 17, pool_blocks=1 << 15, max_returns=1 << 15,
            max_points=1 << 14)
K = 8
TAU_S = 0.005


@pytest.fixture(scope="module")
def scene():
    import torch
    W = workload.single_frame()
    fr, pts, nrm = workload.single_frame_inputs(W)
    g = af.Map(W.af_config(**CAPS))
    g.set_tool(W.af_tool(), W.dirs)
    g.integrate_scan(to_dev(fr.pts), fr.pose)
    om = oracle.Map(oracle_config(W))
    om.integrate(fr.pts, fr.pose)
    torch.cuda.synchronize()
    rng = np.random.default_rng(21)
    idx = rng.choice(len(pts), 300, replace=False)
    P = pts[idx].copy()
    N = nrm[idx].copy()
    # edge cases: a point far outside the box, normals on the -z / +z branches
    P[-1] = [50.0, 50.0, 50.0]
    N[-2] = [0.0, 0.0, -1.0]
    N[-3] = [0.0, 0.0, 1.0]
    table = synth.fibonacci_hemisphere(K)
    u0 = oracle.soft_seed(N, table)
    n = len(u0)
    al = rng.uniform(-0.3, 0.3, n).astype(np.float32)
    be = rng.uniform(-0.3, 0.3, n).astype(np.float32)
    h = rng.uniform(0.0, 0.03, n).astype(np.float32)
    al[5] = np.nan                         # a non-finite input
    return W, fr, g, om, P, N, table, u0, al, be, h


def _gpu(x):
    return to_dev(np.ascontiguousarray(x, np.float32))


def test_seed_bit_exact(scene):
    W, fr, g, om, P, N, table, u0, *_ = scene
    got = g.soft_seed(_gpu(N), table).cpu().numpy()
    np.testing.assert_array_equal(got, u0)


def test_clearance_matches_oracle(scene):
    import torch
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    cmin = torch.empty(len(u0), dtype=torch.float32, device="cuda")
    c = g.soft_clearance_raw(_gpu(P), _gpu(u0), _gpu(al), _gpu(be), _gpu(h), K, TAU_S,
                             cmin=cmin).cpu().numpy()
    ref, _ = om.soft_clearance(oracle_tool(W), P, K, u0, al, be, h, TAU_S)
    ref_min = om.last_cmin
    assert np.isnan(c[5]) and np.isnan(ref[5])
    ok = ~np.isnan(ref)
    assert np.isfinite(c[ok]).all()
    np.testing.assert_allclose(c[ok], ref[ok], rtol=0, atol=1e-5)
    np.testing.assert_allclose(cmin.cpu().numpy()[ok], ref_min[ok], rtol=0, atol=1e-5)
    # the far point reads tau everywhere: the unobserved closed form
    far = slice(len(u0) - K, len(u0))
    assert np.ptp(c[far]) == 0
    # both signs of the hard clearance occur in this scene
    assert (ref_min[ok] > 0).any() and (ref_min[ok] < 0).any()


def test_adjoint_matches_oracle_gradient(scene):
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    rng = np.random.default_rng(22)
    gc = rng.uniform(0.5, 2.0, len(u0)).astype(np.float32)
    c, ga, gb, gh = (t.cpu().numpy() for t in g.soft_clearance_adjoint(
        _gpu(P), _gpu(u0), _gpu(al), _gpu(be), _gpu(h), K, TAU_S, _gpu(gc)))
    ref_c, ref_g = om.soft_clearance(oracle_tool(W), P, K, u0, al, be, h, TAU_S)
    ok = ~np.isnan(ref_c)
    np.testing.assert_allclose(c[ok], ref_c[ok], rtol=0, atol=1e-5)
    for k, got in enumerate((ga, gb, gh)):
        want = gc.astype(np.float64) * ref_g[:, k]
        err = np.abs(got[ok] - want[ok]) / np.maximum(np.abs(want[ok]), 1e-2)
        assert err.max() <= 1e-3, (k, err.max())
    assert np.isnan(ga[5]) and np.isnan(gb[5]) and np.isnan(gh[5])
    assert (np.abs(ref_g[ok]).max(1) > 0.05).mean() > 0.2      # gradients are not trivial


def test_adjoint_matches_central_differences(scene):
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    tool = oracle_tool(W)
    ok = np.isfinite(al)
    _, ga, gb, gh = (t.cpu().numpy() for t in g.soft_clearance_adjoint(
        _gpu(P), _gpu(u0), _gpu(al), _gpu(be), _gpu(h), K, TAU_S))
    _, ref_g = om.soft_clearance(tool, P, K, u0, al, be, h, TAU_S)
    step = np.float32(1e-4)
    smooth_total = 0
    for k, grad in enumerate((ga, gb, gh)):
        up = [al.copy(), be.copy(), h.copy()]
        dn = [al.copy(), be.copy(), h.copy()]
        up[k] += step
        dn[k] -= step
        cp = g.soft_clearance_raw(_gpu(P), _gpu(u0), *(_gpu(x) for x in up), K, TAU_S).cpu().numpy()
        cm = g.soft_clearance_raw(_gpu(P), _gpu(u0), *(_gpu(x) for x in dn), K, TAU_S).cpu().numpy()
        width = up[k].astype(np.float64) - dn[k].astype(np.float64)
        fd = (cp.astype(np.float64) - cm.astype(np.float64)) / width
        # the oracle, in double, tells where the interval holds no kink
        ocp, _ = om.soft_clearance(tool, P, K, u0, *up, TAU_S)
        ocm, _ = om.soft_clearance(tool, P, K, u0, *dn, TAU_S)
        ofd = (ocp - ocm) / width
        smooth = ok & (np.abs(ofd - ref_g[:, k]) <= 1e-4 * np.maximum(np.abs(ref_g[:, k]), 1e-2))
        assert smooth.mean() > 0.8
        gs = grad[smooth].astype(np.float64)
        d = fd[smooth] - gs
        rel = np.linalg.norm(d) / np.linalg.norm(gs)
        assert rel <= 1e-3, (k, rel)
        # per pair: rel. err <= 1e-3 up to what single precision lets a central
        # difference resolve -- the share of the kernel's own rounding of C at
        # the two ends (|C_fp32 - C_fp64| / width, against the oracle) and the
        # double-precision difference's distance from the analytic gradient
        noise = (np.abs(cp.astype(np.float64) - ocp) + np.abs(cm.astype(np.float64) - ocm)) / width
        resid = np.abs(ofd - ref_g[:, k])
        bound = 1e-3 * np.abs(gs) + noise[smooth] + resid[smooth]
        worst = np.argmax(np.abs(d) - bound)
        assert (np.abs(d) <= bound).all(), (k, d[worst], gs[worst], noise[smooth][worst])
        # where the difference itself is good to 1e-3 (|grad| >= 1e3 x its
        # error), the two agree to the bar plus that error
        big = 1e-3 * np.abs(gs) >= noise[smooth] + resid[smooth]
        assert big.sum() >= 50, (k, big.sum())
        assert (np.abs(d[big]) <= 2e-3 * np.abs(gs[big])).all(), k
        smooth_total += smooth.sum()
    assert smooth_total > 0.8 * 3 * ok.sum()


def test_autograd_function_equals_adjoint(scene):
    import torch
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    sel = np.isfinite(al)
    a = _gpu(np.where(sel, al, 0)).requires_grad_()
    b = _gpu(be).requires_grad_()
    hh = _gpu(h).requires_grad_()
    w = torch.linspace(0.5, 1.5, len(u0), device="cuda")
    C = g.soft_clearance(_gpu(P), _gpu(u0), a, b, hh, K, TAU_S)
    (C * w).sum().backward()
    _, ga, gb, gh = g.soft_clearance_adjoint(_gpu(P), _gpu(u0), a.detach(), b.detach(),
                                             hh.detach(), K, TAU_S, w.contiguous())
    assert torch.equal(a.grad, ga) and torch.equal(b.grad, gb) and torch.equal(hh.grad, gh)
    # only alpha requiring grad: the others get none
    a2 = a.detach().clone().requires_grad_()
    g.soft_clearance(_gpu(P), _gpu(u0), a2, b.detach(), hh.detach(), K, TAU_S).sum().backward()
    assert torch.equal(a2.grad, g.soft_clearance_adjoint(
        _gpu(P), _gpu(u0), a.detach(), b.detach(), hh.detach(), K, TAU_S)[1])


def test_refine_and_best(scene):
    import torch
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    tool = oracle_tool(W)
    z = np.zeros(len(u0), np.float32)
    # steps = 0 is the forward pass, bit for bit
    a0, b0, h0 = _gpu(z), _gpu(z), _gpu(z)
    c0, m0 = g.soft_refine(_gpu(P), _gpu(u0), a0, b0, h0, K, steps=0)
    cmin = torch.empty(len(u0), dtype=torch.float32, device="cuda")
    cf = g.soft_clearance_raw(_gpu(P), _gpu(u0), _gpu(z), _gpu(z), _gpu(z), K, TAU_S, cmin=cmin)
    assert torch.equal(c0, cf) and torch.equal(m0, cmin)
    # 20 steps in one launch == 20 launches of one step
    lr = dict(lr_dir=0.05, lr_h=0.005, h_max=0.05)
    A, B, H = _gpu(z), _gpu(z), _gpu(z)
    c20, m20 = g.soft_refine(_gpu(P), _gpu(u0), A, B, H, K, steps=20, **lr)
    A1, B1, H1 = _gpu(z), _gpu(z), _gpu(z)
    for _ in range(20):
        c1, m1 = g.soft_refine(_gpu(P), _gpu(u0), A1, B1, H1, K, steps=1, **lr)
    c1, m1 = g.soft_refine(_gpu(P), _gpu(u0), A1, B1, H1, K, steps=0, **lr)
    for x, y in ((A, A1), (B, B1), (H, H1), (c20, c1), (m20, m1)):
        assert torch.equal(x, y)
    assert (H >= 0).all() and (H <= np.float32(0.05)).all()
    # against the oracle's trajectories: equal to rounding except where a
    # trajectory meets a kink of trilinear interpolation within rounding
    ra, rb, rh, rc, rm = om.soft_refine(tool, P, K, u0, z, z, z, 20, **lr)
    dc = np.abs(c20.cpu().numpy() - rc)
    assert (dc <= 1e-5).mean() >= 0.99, np.sort(dc)[-10:]
    assert (np.abs(m20.cpu().numpy() - rm) <= 1e-5).mean() >= 0.99
    gain = c20.cpu().numpy() - c0.cpu().numpy()
    assert gain.mean() > 0 and (gain >= -1e-3).mean() > 0.99
    # per point best of the final C: first maximum, NaN-free
    bk, bc, bu = g.soft_best(c20, K, _gpu(u0))
    cc = c20.cpu().numpy().reshape(-1, K)
    np.testing.assert_array_equal(bk.cpu().numpy(), cc.argmax(1))
    np.testing.assert_array_equal(bc.cpu().numpy(), cc.max(1))
    np.testing.assert_array_equal(bu.cpu().numpy(), u0.reshape(-1, K, 3)[np.arange(len(cc)),
                                                                        cc.argmax(1)])


def test_best_ties_nan_and_ragged():
    import torch
    W = workload.single_frame()
    g = af.Map(W.af_config(**CAPS))
    c = torch.tensor([1.0, 3.0, 3.0, float("nan"), float("nan"), float("nan"), 2.0],
                     device="cuda")
    u0 = torch.arange(21, dtype=torch.float32, device="cuda").reshape(7, 3)
    bk, bc, bu = g.soft_best(c, 3, u0)
    assert bk.tolist() == [1, -1, 0]          # lowest index of the maximum; all NaN; ragged
    assert bc[0].item() == 3.0 and np.isnan(bc[1].item()) and bc[2].item() == 2.0
    assert bu[0].tolist() == [3.0, 4.0, 5.0] and torch.isnan(bu[1]).all()


def test_views_follow_new_scans(scene):
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    W2 = workload.single_frame(seed=77)
    fr2, _, _ = workload.single_frame_inputs(W2, 8000)
    m1 = af.Map(W.af_config(**CAPS))
    m1.set_tool(W.af_tool(), W.dirs)
    o1 = oracle.Map(oracle_config(W))
    m1.integrate_scan(to_dev(fr.pts), fr.pose)
    o1.integrate(fr.pts, fr.pose)
    ok = np.isfinite(al)
    before = m1.soft_clearance_raw(_gpu(P), _gpu(u0), _gpu(al), _gpu(be), _gpu(h), K).cpu().numpy()
    m1.integrate_scan(to_dev(fr2.pts), fr2.pose)
    o1.integrate(fr2.pts, fr2.pose)
    after = m1.soft_clearance_raw(_gpu(P), _gpu(u0), _gpu(al), _gpu(be), _gpu(h), K).cpu().numpy()
    ref, _ = o1.soft_clearance(oracle_tool(W), P, K, u0, al, be, h, TAU_S)
    np.testing.assert_allclose(after[ok], ref[ok], rtol=0, atol=1e-5)
    assert np.abs(after[ok] - before[ok]).max() > 1e-4     # the second scan changed the field


def test_argument_errors(scene):
    import torch
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    bare = af.Map(W.af_config(**CAPS))
    x = _gpu(z := np.zeros(4, np.float32))
    with pytest.raises(af.AfError) as e:
        bare.soft_clearance_raw(_gpu(P[:1]), _gpu(u0[:4]), x, x, x, 4)
    assert e.value.status == af.ERR_STATE
    with pytest.raises(af.AfError) as e:
        g.soft_clearance_raw(_gpu(P[:1]), _gpu(u0[:4]), x, x, x, 4, tau_s=0.0)
    assert e.value.status == af.ERR_INVALID_ARG
    long_excl = af.ToolConfig(**{**W.tool(), "self_excl": 1.3})
    bare.set_tool(long_excl, W.dirs)
    with pytest.raises(af.AfError) as e:
        bare.soft_clearance_raw(_gpu(P[:1]), _gpu(u0[:4]), x, x, x, 4)
    assert e.value.status == af.ERR_STATE
    # no pairs: nothing to do, no error
    e0 = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    e1 = torch.empty(0, dtype=torch.float32, device="cuda")
    assert g.soft_clearance_raw(e0, e0, e1, e1, e1, 4).numel() == 0
    assert g.soft_refine(e0, e0, e1, e1, e1, 4)[0].numel() == 0


def test_start_from_plain_best(scene):
    """Refinement starts from the plain path's result: the best direction of
    each accessible point, NaN (skipped, NaN outputs) for the others."""
    import torch
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    lab, best = g.score(_gpu(P), _gpu(N))
    start = g.soft_start(lab, best).cpu().numpy()
    lab_h, best_h = lab.cpu().numpy(), best.cpu().numpy()
    acc = lab_h == af.ACCESSIBLE
    assert acc.any() and (~acc).any()
    np.testing.assert_array_equal(start[acc], W.dirs[best_h[acc]])
    assert np.isnan(start[~acc]).all()
    z = np.zeros(len(P), np.float32)
    A, B, H = _gpu(z), _gpu(z), _gpu(z)
    c, cmin = g.soft_refine(_gpu(P), _gpu(start), A, B, H, 1, steps=20)
    c = c.cpu().numpy()
    assert np.isnan(c[~acc]).all() and np.isfinite(c[acc]).all()
    assert np.isnan(A.cpu().numpy()[~acc]).all()
    ra, rb, rh, rc, rm = om.soft_refine(oracle_tool(W), P[acc], 1, W.dirs[best_h[acc]],
                                        z[acc], z[acc], z[acc], 20, 0.05, 0.005, 0.05)
    assert (np.abs(c[acc] - rc) <= 1e-5).mean() >= 0.99


def test_sparse_view_equals_dense(scene):
    """The brick-sparse SDF view holds the same corner values as the dense
    one, so clearance, adjoint and refinement are identical bit for bit."""
    import torch
    W, fr, g, om, P, N, table, u0, al, be, h = scene
    g2 = af.Map(W.af_config(**CAPS))
    g2.set_tool(W.af_tool(), W.dirs)
    g2.integrate_scan(to_dev(fr.pts), fr.pose)
    g2.soft_set_view(2)
    g.soft_set_view(1)
    args = (_gpu(P), _gpu(u0), _gpu(al), _gpu(be), _gpu(h), K, TAU_S)
    out = []
    for m in (g, g2):
        c = m.soft_clearance_raw(*args)
        adj = m.soft_clearance_adjoint(*args)
        a2, b2, h2 = _gpu(np.where(np.isfinite(al), al, 0)), _gpu(be), _gpu(h)
        rc, rm = m.soft_refine(_gpu(P), _gpu(u0), a2, b2, h2, K, steps=5)
        out.append([c, *adj, rc, rm, a2, b2, h2])
    for x, y in zip(*out):
        assert torch.equal(torch.nan_to_num(x, nan=7.0), torch.nan_to_num(y, nan=7.0))
    assert g.sync_status() == 0 and g2.sync_status() == 0
    g.soft_set_view(0)
