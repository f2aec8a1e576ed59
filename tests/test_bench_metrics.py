"""Host-side metrics of bench.py's experiments, on CPU.

The relative torque error of Sec. 3 compares the torque X x g of a body
about the coordinate origin with that of the exact direct-sum acceleration.
Pinned by a worked case, by the part of an acceleration error that a torque
cannot see (a component along X), and by rotation invariance."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_torque_error_worked_case():
    # X = e_x, g = e_y, g_PP = 2 e_y: torques e_z and 2 e_z, error 1/2
    e = bench.torque_errors([[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]], [[0.0, 2.0, 0.0]])
    assert float(e[0]) == 0.5


def test_torque_error_blind_to_radial_error():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(64, 3))
    g_ref = rng.normal(size=(64, 3))
    g = g_ref + rng.normal(size=(64, 1)) * x  # an error along X only
    e = bench.torque_errors(x, g, g_ref).numpy()
    assert np.all(e < 1e-12)
    # an error across X shows up in full: |X x d| / |X x g_PP|
    d = np.cross(x, rng.normal(size=(64, 3)))
    e2 = bench.torque_errors(x, g_ref + d, g_ref).numpy()
    want = np.linalg.norm(np.cross(x, d), axis=1) / np.linalg.norm(np.cross(x, g_ref), axis=1)
    assert np.allclose(e2, want, rtol=1e-12)


def test_torque_error_rotation_invariant():
    rng = np.random.default_rng(4)
    x, g, g_ref = (rng.normal(size=(32, 3)) for _ in range(3))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    a = bench.torque_errors(x, g, g_ref).numpy()
    b = bench.torque_errors(x @ q.T, g @ q.T, g_ref @ q.T).numpy()
    assert np.allclose(a, b, rtol=1e-12)
