"""Pins of the reference network (oracle/mlp.py): its gradient against
finite differences in float64, and the bfloat16 rounding against its
definition."""
import numpy as np

from oracle import mlp as M


def _params(seed=0):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=M.NPARAMS) * 0.2
    p[M.NW:M.NW + 8] = rng.normal(size=8)
    p[M.NW + 8:] = rng.uniform(0.5, 2.0, 8)
    return p


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params()
    X = rng.normal(size=(50, 8))
    y = rng.normal(size=50)
    _, g = M.loss_and_grad(p, X, y, "fp64")
    for k in list(range(0, M.NW, 577)) + [M.NW - 1, M.NW - 2]:
        e = np.zeros_like(p)
        e[k] = 1e-6
        fd = (M.loss_and_grad(p + e, X, y, "fp64")[0] - M.loss_and_grad(p - e, X, y, "fp64")[0]) / 2e-6
        assert abs(fd - g[k]) <= 1e-6 * (1 + abs(g[k])), k


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, -3.0, 0.0], dtype=np.float32)
    # the bfloat16 spacing at 1 is 2^-7: 1 + 2^-8 is a tie -> even (1.0); 1 + 2^-9 -> 1.0;
    # 1 + 3 * 2^-9 -> 1 + 2^-7
    assert np.array_equal(M.bf16(x), np.array([1.0, 1.0, 1.0, 1.0078125, -3.0, 0.0], dtype=np.float32))


def test_bf16_form_tracks_fp64_form():
    rng = np.random.default_rng(2)
    p = _params(3)
    X = rng.normal(size=(200, 8))
    y64, _, _ = M.forward(p, X, "fp64")
    y16, _, _ = M.forward(p.astype(np.float32), X.astype(np.float32), "bf16")
    assert np.abs(y64 - y16).max() <= 0.05 * (1 + np.abs(y64).max())
