"""Pins of the oracle's softened Green's function (CPU).

The paper remarks (Sec. 4) that the torque correction applies to any Green's
function that depends only on the distance; the softened form used here is
Plummer's, G(R) = -1/sqrt(R^2 + eps^2).  Its derivative tensors have the same
structure as those of -1/R with R replaced by sqrt(R^2 + eps^2); they are no
longer traceless: the trace of D_ij is the Laplacian of G, 3 eps^2 / (R^2 +
eps^2)^(5/2) (4 pi times the Plummer density of unit mass)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

EPS = 0.3


def _fd(f, r, h=1e-5):
    out = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        out.append((f(r + e) - f(r - e)) / (2 * h))
    return np.stack(out, axis=-1)


@pytest.mark.parametrize("r", [np.array([0.7, -0.4, 1.1]), np.array([0.05, 0.02, -0.03])])
def test_softened_tensors_are_successive_derivatives(r):
    D0, D1, D2, D3, D4, _ = oracle.dtensor_p3(r, EPS)
    R2 = r @ r + EPS ** 2
    assert abs(D0 + 1 / np.sqrt(R2)) < 1e-15 * abs(D0)
    pick = lambda k: (lambda q: np.asarray(oracle.dtensor_p3(q, EPS)[k]))
    assert np.allclose(_fd(pick(0), r), D1, rtol=1e-8, atol=1e-9 * np.abs(D1).max())
    assert np.allclose(_fd(pick(1), r), D2, rtol=1e-7, atol=1e-8 * np.abs(D2).max())
    assert np.allclose(_fd(pick(2), r), D3, rtol=1e-7, atol=1e-8 * np.abs(D3).max())
    assert np.allclose(_fd(pick(3), r), D4, rtol=1e-6, atol=1e-7 * np.abs(D4).max())


def test_softened_trace_is_the_plummer_density():
    rng = np.random.default_rng(1)
    for _ in range(5):
        r = rng.normal(size=3)
        _, _, D2, D3, D4, _ = oracle.dtensor_p3(r, EPS)
        u = r @ r + EPS ** 2
        assert abs(np.trace(D2) - 3 * EPS ** 2 / u ** 2.5) <= 1e-14 * np.abs(D2).max()
        # the trace of a higher derivative is the derivative of the trace
        lap = lambda q: np.array(3 * EPS ** 2 / (q @ q + EPS ** 2) ** 2.5)
        assert np.allclose(np.einsum("ijj->i", D3), _fd(lap, r), rtol=1e-7)
        assert np.allclose(D4, D4.transpose(1, 0, 2, 3)) and np.allclose(D4, D4.transpose(0, 2, 1, 3))


def test_softened_generic_tensors_match_explicit_and_limit():
    r = np.array([0.3, -0.8, 0.5])
    D = oracle.dtensor_p3(r, EPS)
    for n in range(5):
        g = oracle.dtensor_generic(r, n, EPS)
        full = np.asarray(D[n])
        for k, (a, b, c) in enumerate(oracle.multi_indices(n)):
            idx = (0,) * a + (1,) * b + (2,) * c
            assert abs(g[k] - (full[idx] if n else full)) <= 1e-14 * max(1.0, np.abs(full).max())
    # eps -> 0 recovers the paper's 1/R tensors
    for n in range(7):
        assert np.allclose(oracle.dtensor_generic(r, n, 1e-9), oracle.dtensor_generic(r, n), rtol=1e-12)


def test_softened_direct_two_bodies_closed_form():
    # bodies at 0 and (d, 0, 0), masses 2 and 3: a_1 = 3 d / (d^2 + eps^2)^(3/2)
    x = np.array([0.0, 1.5])
    y = z = np.zeros(2)
    m = np.array([2.0, 3.0])
    a = oracle.direct(x, y, z, m, eps=EPS)
    f = 1.5 / (1.5 ** 2 + EPS ** 2) ** 1.5
    assert np.allclose(a, [[3 * f, 0, 0], [-2 * f, 0, 0]], rtol=1e-15, atol=0)


def test_softened_theta_to_zero_is_softened_direct():
    b = ics.plummer(1500, seed=3)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 1e-7, 25, softening=0.05)
    ref = oracle.direct(b.x, b.y, b.z, b.m, eps=0.05)
    a = o.accel("TC")
    assert (np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 1e-13


def _octupole(p, m, Zc):
    x = p - Zc
    return np.einsum("n,ni,nj,nk->ijk", m, x, x, x)


@pytest.mark.parametrize("P", [3, 4, 5])
def test_softened_pair_torque_cancels_and_uc_matches_closed_form(P):
    """Per accepted pair with softening: force balance for every variant; the
    TC and TCO torques at rounding; the UC torque equals
    1/2 eps_piq (M_A O_B - O_A M_B)_pjk D_ijk(r) with the softened D_ijk
    (the net torque equation holds for any radial G) at P = 3."""
    b = ics.plummer(800, seed=12)
    eps = 0.05
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.6, 16, P=P, softening=eps)
    m2l, _, _ = o.lists()
    c = o.cells()
    M, Z, _, _ = o.geometry()
    p = b.pos()
    sel = [k for k in range(len(m2l)) if c.count[m2l[k, 0]] >= 3 and c.count[m2l[k, 1]] >= 3]
    # pairs at separations comparable with eps, where softening matters
    d = np.array([np.linalg.norm(Z[m2l[k, 0]] - Z[m2l[k, 1]]) for k in sel])
    sel = [sel[i] for i in np.argsort(d)[:4]]
    assert d.min() < 10 * eps
    eps3 = np.zeros((3, 3, 3))
    for i, j, k in itertools.permutations(range(3)):
        eps3[i, j, k] = np.linalg.det(np.eye(3)[[i, j, k]])
    for k in sel:
        A, B = m2l[k]
        for v in ("UC", "TC", "TCO"):
            a = o.pair_accel(A, B, v, generic=P > 3)
            f = (b.m[:, None] * a).sum(0)
            t = (b.m[:, None] * np.cross(p, a)).sum(0)
            sc = (b.m[:, None] * np.abs(np.cross(p, a))).sum(0).max()
            assert np.abs(f).max() <= 1e-13 * (b.m[:, None] * np.abs(a)).sum(0).max()
            if v == "UC":
                assert np.abs(t).max() > 1e-10 * sc
                if P == 3:
                    ia, ib = o.cell_bodies(A), o.cell_bodies(B)
                    S = M[A] * _octupole(p[ib], b.m[ib], Z[B]) - _octupole(p[ia], b.m[ia], Z[A]) * M[B]
                    D3 = oracle.dtensor_p3(Z[A] - Z[B], eps)[3]
                    tau = 0.5 * np.einsum("piq,pjk,ijk->q", eps3, S, D3)
                    assert np.allclose(t, tau, rtol=1e-9, atol=1e-12 * sc)
            else:
                assert np.abs(t).max() <= 1e-13 * sc, (P, v)


def test_softened_solve_error_and_balances():
    """A softened solve at theta = 0.5 against the softened direct sum: error
    of the same size as the unsoftened method's, force balance at rounding
    for every variant, torque balance at rounding for TC and TCO only."""
    b = ics.plummer(2000, seed=0)
    eps = 0.02
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25, softening=eps)
    ref = oracle.direct(b.x, b.y, b.z, b.m, eps=eps)
    res = {}
    for v in ("UC", "TC", "TCO"):
        a = o.accel(v)
        res[v] = (oracle.balance(b.x, b.y, b.z, b.m, a), oracle.force_errors(a, ref)["rms"])
    assert res["TC"][1] < 1e-2
    for v in res:
        assert res[v][0][0] < 1e-15
    assert res["TC"][0][1] < 1e-15 and res["TCO"][0][1] < 1e-15
    assert res["UC"][0][1] > 1e3 * res["TC"][0][1]
