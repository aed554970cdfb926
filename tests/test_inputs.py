"""The seeded input generators' direction tables: the Fibonacci sets of the
workloads and the paper's approach set (Sec. 3.4: D = 180 yaw angles over
[0, 2 pi) at a fixed, horizontal pitch, with a 70 degree normal cone)."""
import math

import numpy as np

from paper_2608_06412_gb300 import synth


def test_yaw_ring_is_the_horizontal_ring_in_yaw_order():
    u = synth.yaw_ring(180).astype(np.float64)
    assert u.shape == (180, 3) and u.dtype == np.float64
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-7)
    assert (u[:, 2] == 0.0).all()                        # pitch 0: horizontal
    yaw = np.mod(np.arctan2(u[:, 1], u[:, 0]), 2 * math.pi)
    np.testing.assert_allclose(np.diff(yaw), 2 * math.pi / 180, atol=1e-6)
    assert abs(yaw[0]) < 1e-7                            # psi_0 = 0, increasing
    # a pitched ring keeps the yaw order and lifts every direction equally
    p = synth.yaw_ring(36, pitch=0.3).astype(np.float64)
    np.testing.assert_allclose(p[:, 2], math.sin(0.3), atol=1e-7)


def test_seventy_degree_cone():
    assert synth.COS_70 == float(np.float32(math.cos(math.radians(70.0))))
    # a horizontal normal keeps the ring directions within 70 degrees: 69 of 180
    # (yaw offsets -68 .. +68 degrees in steps of 2)
    u = synth.yaw_ring(180)
    n = np.array([1.0, 0.0, 0.0], np.float32)
    assert int((u @ n > np.float32(synth.COS_70)).sum()) == 69


def test_fibonacci_sets():
    d = synth.fibonacci_dirs(128).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    # equal-area bands: z_i = 1 - (2i + 1) / G
    np.testing.assert_allclose(d[:, 2], 1.0 - (2.0 * np.arange(128) + 1.0) / 128, atol=1e-7)
    assert abs(d.mean(0)).max() < 0.02                   # balanced over the sphere
    h = synth.fibonacci_hemisphere(64).astype(np.float64)
    assert (h[:, 2] > 0).all() and abs(np.linalg.norm(h, axis=1) - 1).max() < 1e-6
