"""Pins of the oracle's soft clearance (the differentiable form) against what
mathematics fixes, independently of the oracle's own formulas:

* trilinear interpolation reproduces a linear field exactly, so on a map whose
  voxels hold a linear function the sampled SDF is that function at the
  sample points; C is then the softmin of closed-form values, and its
  gradient the derivative of that closed form, taken here by finite
  differences in double precision;
* softmin tends to the plain minimum as tau_s -> 0;
* an unobserved map reads tau everywhere: closed-form C, zero gradient;
* on a real integrated scene the analytic gradient equals central finite
  differences of the oracle's own C wherever no sample crosses a cell face
  inside the difference interval;
* the seed frame is orthonormal and right-handed and maps the table's +z to
  the normal exactly.
Parity status: pinned.
"""
import numpy as np
import pytest

import oracle
from paper_2608_06412_gb300 import synth, workload

Q = 2.0 ** 20
V = np.float32(0.02)
TAU = np.float32(0.06)


def _tool(**kw):
    base = dict(radius=0.04, length=0.10, self_excl=0.04, corr_radius=0.05,
                corr_length=0.10, cos_theta_max=0.0, n_c=5, strict=0)
    base.update(kw)
    return oracle.Tool(**base)


def _cfg():
    return oracle.Config(v=float(V), tau=float(TAU), r_c=float(V) / 2, cube_radius=3,
                         clear_samples=8, dom_min=(-64,) * 3, dom_size=(128,) * 3)


def _frame(u0):
    """(t1, t2) of a unit vector, read back through the seed: the table rows
    (1,0,0) and (0,1,0) map to t1 and t2."""
    tab = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    s = oracle.soft_seed(np.asarray(u0, np.float32)[None], tab).astype(np.float64)
    return s[0], s[1], s[2]


def _samples(tool):
    """(j, margin) of every axis sample, decided in single precision."""
    J = int(np.floor(np.float32(np.float32(tool.length) + np.float32(tool.corr_length)) / V))
    out = []
    for j in range(1, J + 1):
        a = np.float32(j) * V
        if not a > np.float32(tool.self_excl):
            continue
        out.append((j, float(np.float32(tool.radius)) if a <= np.float32(tool.length)
                    else float(np.float32(tool.corr_radius))))
    return out


def _softmin(phi, tau_s):
    m = phi.min()
    return m - tau_s * np.log(np.exp(-(phi - m) / tau_s).sum())


# a linear field D(x) = b + a . x, positive over the box used below
A_LIN = np.array([0.31, -0.22, 0.47])
B_LIN = 1.5


@pytest.fixture(scope="module")
def linear_map():
    mp = oracle.Map(_cfg())
    ax = np.arange(-30, 31)
    ijk = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    c = (ijk + 0.5) * np.float64(V)
    d = B_LIN + c @ A_LIN
    assert d.min() > 0
    mp.set_voxels(ijk, np.rint(d * Q).astype(np.uint64), 1)
    return mp


def _closed_form(s, u0, al, be, h, tool, tau_s):
    t1, t2, _ = _frame(u0)
    q = np.asarray(u0, np.float64) + al * t1 + be * t2
    u = q / np.linalg.norm(q)
    phi = []
    for j, margin in _samples(tool):
        x = np.asarray(s, np.float64) + (h + j * np.float64(V)) * u
        phi.append(B_LIN + x @ A_LIN - margin)
    return _softmin(np.array(phi), tau_s), np.array(phi)


def _pairs(rng, n):
    s = rng.uniform(-0.05, 0.05, (n, 3)).astype(np.float32)
    u0 = rng.normal(size=(n, 3))
    u0 /= np.linalg.norm(u0, axis=1, keepdims=True)
    u0 = u0.astype(np.float32)
    ab = rng.uniform(-0.3, 0.3, (n, 2)).astype(np.float32)
    h = rng.uniform(0.0, 0.05, n).astype(np.float32)
    return s, u0, ab, h


def test_linear_field_value_and_gradient(linear_map):
    rng = np.random.default_rng(5)
    tool = _tool()
    tau_s = 0.005
    s, u0, ab, h = _pairs(rng, 24)
    for fp32 in (True, False):
        c, g = linear_map.soft_clearance(tool, s, 1, u0, ab[:, 0], ab[:, 1], h, tau_s, fp32)
        for i in range(len(s)):
            al, be, hh = (float(x) for x in (ab[i, 0], ab[i, 1], h[i]))
            ref, _ = _closed_form(s[i], u0[i], al, be, hh, tool, tau_s)
            # voxel values carry 2^-20 quantisation and single-precision rounding
            assert abs(c[i] - ref) < 3e-6, (i, c[i], ref)
            eps = 1e-5
            fd = []
            for k in range(3):
                p = [al, be, hh]
                m = [al, be, hh]
                p[k] += eps
                m[k] -= eps
                fd.append((_closed_form(s[i], u0[i], *p, tool, tau_s)[0]
                           - _closed_form(s[i], u0[i], *m, tool, tau_s)[0]) / (2 * eps))
            fd = np.array(fd)
            np.testing.assert_allclose(g[i], fd, rtol=2e-3, atol=2e-4 * np.abs(A_LIN).sum())


def test_softmin_tends_to_minimum(linear_map):
    rng = np.random.default_rng(6)
    tool = _tool()
    s, u0, ab, h = _pairs(rng, 8)
    c, _ = linear_map.soft_clearance(tool, s, 1, u0, ab[:, 0], ab[:, 1], h, 1e-7)
    cmin = linear_map.last_cmin
    for i in range(len(s)):
        _, phi = _closed_form(s[i], u0[i], float(ab[i, 0]), float(ab[i, 1]), float(h[i]),
                              tool, 0.005)
        assert abs(c[i] - phi.min()) < 3e-6
        assert abs(cmin[i] - phi.min()) < 3e-6      # the hard clearance
    # and C never exceeds the minimum: softmin is a lower bound of min
    c2, _ = linear_map.soft_clearance(tool, s, 1, u0, ab[:, 0], ab[:, 1], h, 0.02)
    assert (c2 <= c + 1e-12).all()


def test_unobserved_map_reads_tau():
    mp = oracle.Map(_cfg())
    tool = _tool(length=0.25, corr_length=1.0)
    rng = np.random.default_rng(7)
    s, u0, ab, h = _pairs(rng, 10)
    tau_s = 0.005
    c, g = mp.soft_clearance(tool, s, 1, u0, ab[:, 0], ab[:, 1], h, tau_s)
    phi = np.array([float(TAU) - m for _, m in _samples(tool)])
    np.testing.assert_allclose(c, _softmin(phi, tau_s), rtol=0, atol=1e-12)
    assert (g == 0).all()
    # samples that leave the map box read tau as well
    far = np.full((1, 3), 1.27, np.float32)     # the box ends at 1.28 m
    c_far, g_far = mp.soft_clearance(tool, far, 1, u0[:1], ab[:1, 0], ab[:1, 1], h[:1], tau_s)
    assert c_far[0] == pytest.approx(_softmin(phi, tau_s), abs=1e-12) and (g_far == 0).all()


def test_seed_frame_is_orthonormal():
    rng = np.random.default_rng(8)
    n = rng.normal(size=(200, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n = np.concatenate([n, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 0, -0.0]]])
    n[-1] = [0.6, 0.8, -0.0]
    n = n.astype(np.float32)
    for k in range(len(n)):
        t1, t2, z = _frame(n[k])
        assert (z == n[k].astype(np.float64)).all()     # +z maps to the normal exactly
        for a, b in ((t1, t2), (t1, z), (t2, z)):
            assert abs(a @ b) < 1e-6
        assert abs(np.linalg.norm(t1) - 1) < 1e-6 and abs(np.linalg.norm(t2) - 1) < 1e-6
        np.testing.assert_allclose(np.cross(t1, t2), z, atol=1e-6)    # right-handed


def _single_frame_map():
    W = workload.single_frame()
    p = W.params
    cfg = oracle.Config(v=p["v"], tau=p["tau"], r_c=p["r_c"], cube_radius=p["cube_radius"],
                        clear_samples=p["clear_samples"], cone_cos=p["cone_cos"],
                        range_min=p["range_min"], range_max=p["range_max"],
                        clear_lo=p["clear_lo"], clear_hi=p["clear_hi"], w_min=p["w_min"],
                        w_cap=p["w_cap"],
                        dom_min=tuple(8 * b for b in W.dom_min),
                        dom_size=tuple(8 * b for b in W.dom_bricks))
    mp = oracle.Map(cfg)
    fr, pts, nrm = workload.single_frame_inputs(W, 6000)
    mp.integrate(fr.pts, fr.pose)
    return W, mp, pts, nrm


@pytest.fixture(scope="module")
def scene():
    return _single_frame_map()


def test_gradient_matches_finite_differences_on_a_scene(scene):
    W, mp, pts, nrm = scene
    t = W.tool()
    tool = oracle.Tool(radius=t["radius"], length=t["length"], self_excl=t["self_excl"],
                       corr_radius=t["corr_radius"], corr_length=t["corr_length"])
    rng = np.random.default_rng(9)
    idx = rng.choice(len(pts), 40, replace=False)
    table = synth.fibonacci_hemisphere(4)
    u0 = oracle.soft_seed(nrm[idx], table)
    n = len(u0)
    al = rng.uniform(-0.2, 0.2, n).astype(np.float32)
    be = rng.uniform(-0.2, 0.2, n).astype(np.float32)
    h = rng.uniform(0.0, 0.02, n).astype(np.float32)
    tau_s = 0.005
    # exact cells in double: a piecewise-trilinear function of (alpha, beta, h)
    # (the inputs stay single precision; the differences are taken on doubles
    # passed through the float interface, so steps are multiples of the ulp)
    c0, g = mp.soft_clearance(tool, pts[idx], 4, u0, al, be, h, tau_s, fp32_cells=False)
    assert np.isfinite(c0).all() and (np.abs(g).max(1) > 0).mean() > 0.5
    checked = 0
    for k, base in enumerate((al, be, h)):
        fds = []
        for eps in (2.0 ** -20, 2.0 ** -21):
            up, dn = base.copy(), base.copy()
            up += np.float32(eps)
            dn -= np.float32(eps)
            st = [al, be, h]
            st[k] = up
            cp, _ = mp.soft_clearance(tool, pts[idx], 4, u0, *st, tau_s, fp32_cells=False)
            st[k] = dn
            cm, _ = mp.soft_clearance(tool, pts[idx], 4, u0, *st, tau_s, fp32_cells=False)
            fds.append((cp - cm) / (up.astype(np.float64) - dn.astype(np.float64)))
        fd1, fd2 = fds
        scale = np.maximum(np.abs(g[:, k]), 1e-3)
        smooth = np.abs(fd1 - fd2) < 1e-6 * scale      # no cell face crossed
        assert smooth.mean() > 0.7
        err = np.abs(fd1 - g[:, k]) / scale
        assert err[smooth].max() < 1e-5, (k, err[smooth].max())
        checked += smooth.sum()
    assert checked > 80


def test_refine_raises_clearance(scene):
    W, mp, pts, nrm = scene
    t = W.tool()
    tool = oracle.Tool(radius=t["radius"], length=t["length"], self_excl=t["self_excl"],
                       corr_radius=t["corr_radius"], corr_length=t["corr_length"])
    rng = np.random.default_rng(10)
    idx = rng.choice(len(pts), 30, replace=False)
    u0 = oracle.soft_seed(nrm[idx], synth.fibonacci_hemisphere(4))
    n = len(u0)
    z = np.zeros(n, np.float32)
    c0, _ = mp.soft_clearance(tool, pts[idx], 4, u0, z, z, z)
    a, b, h, c, cmin = mp.soft_refine(tool, pts[idx], 4, u0, z, z, z, 20, 0.02, 0.002, 0.05)
    assert (c <= cmin).all()
    assert (h >= 0).all() and (h <= np.float32(0.05)).all()
    # plain gradient ascent with a small step: clearance does not drop (beyond
    # the kinks of trilinear interpolation) and rises on average
    assert (c >= c0 - 1e-3).mean() > 0.95
    assert (c - c0).mean() > 0


def test_single_precision_cells_agree_with_exact_cells(scene):
    """Deciding each sample's cell in single precision (as the kernel does)
    changes nothing but the cells of samples within rounding of a face: C
    agrees to rounding everywhere, the gradient on almost every pair."""
    W, mp, pts, nrm = scene
    t = W.tool()
    tool = oracle.Tool(radius=t["radius"], length=t["length"], self_excl=t["self_excl"],
                       corr_radius=t["corr_radius"], corr_length=t["corr_length"])
    rng = np.random.default_rng(11)
    idx = rng.choice(len(pts), 200, replace=False)
    u0 = oracle.soft_seed(nrm[idx], synth.fibonacci_hemisphere(8))
    n = len(u0)
    al = rng.uniform(-0.2, 0.2, n).astype(np.float32)
    be = rng.uniform(-0.2, 0.2, n).astype(np.float32)
    h = rng.uniform(0.0, 0.02, n).astype(np.float32)
    c32, g32 = mp.soft_clearance(tool, pts[idx], 8, u0, al, be, h, 0.005, fp32_cells=True)
    c64, g64 = mp.soft_clearance(tool, pts[idx], 8, u0, al, be, h, 0.005, fp32_cells=False)
    assert np.abs(c32 - c64).max() < 1e-7
    scale = np.maximum(np.abs(g64), 1e-3)
    same = (np.abs(g32 - g64) < 1e-4 * scale).all(1)
    assert same.mean() > 0.98
