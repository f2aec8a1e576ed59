"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, finite differences, brute force, invariants stated by the paper, or
special cases that reduce to direct summation.  The planted-mistake tests at
the end show that the pins catch a dropped term or a wrong sign.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------
# derivative tensors of G = -1/R (Sec. 2: D, D_i, D_ij, D_ijk; D_ijkl derived)
# ---------------------------------------------------------------------------
def _fd(f, r, h=1e-5):
    """Central differences of f (array-valued) along each axis: out[..., l]."""
    cols = []
    for l in range(3):
        e = np.zeros(3)
        e[l] = h
        cols.append((f(r + e) - f(r - e)) / (2 * h))
    return np.stack(cols, axis=-1)


@pytest.mark.parametrize("r", [np.array([0.7, -1.1, 0.4]), np.array([2.0, 0.3, -0.9]),
                               np.array([-0.2, 0.5, 1.6])])
def test_dtensors_are_successive_derivatives(r):
    D0, D1, D2, D3, D4, _ = oracle.dtensor_p3(r)
    # G = -1/R itself
    assert np.isclose(D0, -1.0 / np.linalg.norm(r), rtol=1e-15)
    pick = lambda k: (lambda q: oracle.dtensor_p3(q)[k])
    scale = np.linalg.norm(r)
    assert np.allclose(_fd(lambda q: np.array(oracle.dtensor_p3(q)[0]), r), D1, rtol=1e-8, atol=1e-9)
    assert np.allclose(_fd(pick(1), r), D2, rtol=1e-7, atol=1e-8 / scale)
    assert np.allclose(_fd(pick(2), r), D3, rtol=1e-7, atol=1e-8 / scale ** 2)
    assert np.allclose(_fd(pick(3), r), D4, rtol=1e-6, atol=1e-7 / scale ** 3)


def test_dtensors_symmetric_and_traceless():
    r = np.array([0.3, -0.8, 1.2])
    _, _, D2, D3, D4, _ = oracle.dtensor_p3(r)
    for T in (D2, D3, D4):
        for p in itertools.permutations(range(T.ndim)):
            assert np.allclose(T, np.transpose(T, p), rtol=1e-14, atol=0)
    # harmonic: -1/R solves Laplace's equation away from the origin
    assert abs(np.trace(D2)) < 1e-14 * np.abs(D2).max()
    assert np.abs(np.einsum("iik->k", D3)).max() < 1e-14 * np.abs(D3).max()
    assert np.abs(np.einsum("iikl->kl", D4)).max() < 1e-14 * np.abs(D4).max()


def test_dprime_keeps_only_torque_terms():
    """D' (Eq. 8) differs from D_ijkl only by terms carrying r_i, so
    r x (D - D') S = 0 for any symmetric S."""
    r = np.array([0.9, 0.2, -0.5])
    _, _, _, _, D4, D4p = oracle.dtensor_p3(r)
    S = np.random.default_rng(0).normal(size=(3, 3, 3))
    S = sum(np.transpose(S, p) for p in itertools.permutations(range(3)))
    diff = np.einsum("ijkl,jkl->i", D4 - D4p, S)
    assert np.linalg.norm(np.cross(r, diff)) < 1e-13 * np.linalg.norm(diff)
    assert np.linalg.norm(diff) > 1e-3  # D' really differs


def test_generic_derivatives_match_explicit_and_fd():
    r = np.array([0.6, -0.7, 1.1])
    D = oracle.dtensor_p3(r)
    for n in range(0, 5):
        g = oracle.dtensor_generic(r, n)
        for k, (a, b, c) in enumerate(oracle.multi_indices(n)):
            idx = (0,) * a + (1,) * b + (2,) * c
            ref = D[0] if n == 0 else D[n][idx]
            assert np.isclose(g[k], ref, rtol=1e-13, atol=1e-15), (n, a, b, c)
    # orders 5 and 6 against finite differences of the order below
    for n in (5, 6):
        lower = {mi: k for k, mi in enumerate(oracle.multi_indices(n - 1))}
        g = oracle.dtensor_generic(r, n)
        for k, (a, b, c) in enumerate(oracle.multi_indices(n)):
            # differentiate the component with one index removed
            if a > 0:
                base, ax = (a - 1, b, c), 0
            elif b > 0:
                base, ax = (a, b - 1, c), 1
            else:
                base, ax = (a, b, c - 1), 2
            h = 1e-5
            e = np.zeros(3)
            e[ax] = h
            fd = (oracle.dtensor_generic(r + e, n - 1)[lower[base]] -
                  oracle.dtensor_generic(r - e, n - 1)[lower[base]]) / (2 * h)
            assert np.isclose(g[k], fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())


# ---------------------------------------------------------------------------
# direct summation (Sec. 3: the reference of the error metric)
# ---------------------------------------------------------------------------
def _golden_bodies(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_direct_closed_forms():
    """Hand-computed accelerations (tests/golden/closed_forms.txt)."""
    data = _golden_bodies("closed_forms.txt")
    for case in np.unique(data[:, 0]):
        d = data[data[:, 0] == case]
        x, y, z, m = d[:, 1], d[:, 2], d[:, 3], d[:, 4]
        a = oracle.direct(x, y, z, m)
        assert np.allclose(a, d[:, 5:8], rtol=1e-14, atol=1e-14), case


def test_direct_matches_pairwise_sum_and_newton_third_law():
    b = ics.uniform_cube(300, seed=3, mass_spread=True)
    a = oracle.direct(b.x, b.y, b.z, b.m)
    p = b.pos()
    d = p[None, :, :] - p[:, None, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    ref = np.einsum("ijk,j->ik", d / r[:, :, None] ** 3, b.m)
    assert np.allclose(a, ref, rtol=1e-12, atol=0)
    tot = (b.m[:, None] * a).sum(0)
    assert np.abs(tot).max() < 1e-13 * np.abs(b.m[:, None] * a).sum(0).max()


# ---------------------------------------------------------------------------
# Morton keys and the octree (Sec. 2)
# ---------------------------------------------------------------------------
def test_morton_keys_by_bit_loops():
    b = ics.plummer(500, seed=1)
    keys, lo, scale = oracle.morton(b.x, b.y, b.z)
    p = b.pos()
    assert np.array_equal(lo, p.min(0))
    ext = (p.max(0) - p.min(0)).max()
    assert scale == 2.0 ** 21 / ext
    for i in range(0, 500, 7):
        q = [min(int(np.floor((p[i, d] - lo[d]) * scale)), 2 ** 21 - 1) for d in range(3)]
        k = 0
        for bit in range(21):
            for d in range(3):
                k |= ((q[d] >> bit) & 1) << (3 * bit + d)
        assert int(keys[i]) == k


def _tree_invariants(o):
    key, order, lo, scale = o.keys()
    c = o.cells()
    n = o.n
    assert np.all(np.diff(key.astype(np.float64)) >= 0)
    assert np.array_equal(np.sort(order), np.arange(n))
    # sorted by (key, caller index)
    kk = key.astype(object)
    for s in range(1, n):
        assert (kk[s - 1], order[s - 1]) < (kk[s], order[s])
    # breadth-first numbering: level-major, begin ascending within a level
    assert np.all(np.diff(c.level) >= 0)
    for lev in np.unique(c.level):
        sel = np.where(c.level == lev)[0]
        assert np.all(np.diff(c.begin[sel]) > 0)
    for cid in range(o.ncell):
        b, cnt, lev = c.begin[cid], c.count[cid], c.level[cid]
        assert cnt >= 1
        # all bodies share the first `lev` octal digits of the key
        shift = 3 * (21 - lev)
        pre = key[b:b + cnt] >> np.uint64(shift) if lev > 0 else np.zeros(cnt, np.uint64)
        assert np.all(pre == pre[0])
        if c.nchild[cid] == 0:
            assert cnt <= o.n_crit or lev == 21
        else:
            assert cnt > o.n_crit
            f, k = c.first_child[cid], c.nchild[cid]
            kids = np.arange(f, f + k)
            assert np.all(c.parent[kids] == cid)
            assert c.begin[f] == b
            assert np.sum(c.count[kids]) == cnt
            assert np.all(c.begin[kids[1:]] == c.begin[kids[:-1]] + c.count[kids[:-1]])
    return c


def test_tree_structure_invariants():
    b = ics.plummer(3000, seed=2)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _tree_invariants(o)


def test_tree_with_coincident_bodies_reaches_depth_cap():
    p = np.concatenate([np.zeros((30, 3)), np.random.default_rng(1).uniform(-1, 1, (200, 3))])
    m = np.ones(p.shape[0])
    o = oracle.Oracle(p[:, 0], p[:, 1], p[:, 2], m, 0.5, 25)
    c = _tree_invariants(o)
    assert c.level.max() == 21
    deep = np.where((c.level == 21) & (c.nchild == 0))[0]
    assert np.any(c.count[deep] >= 30)


def test_centre_of_mass_rmax_and_moments_by_definition():
    b = ics.uniform_cube(2000, seed=4, mass_spread=True)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25, P=3)
    key, order, _, _ = o.keys()
    c = o.cells()
    M, Z, R, mom = o.geometry()
    p, m = b.pos()[order], b.m[order]
    mi = [oracle.multi_indices(n) for n in range(4)]
    flat = [t for grp in mi for t in grp]
    for cid in range(0, o.ncell, 3):
        s = slice(c.begin[cid], c.begin[cid] + c.count[cid])
        pc, mc = p[s], m[s]
        Mc = mc.sum()
        Zc = (mc[:, None] * pc).sum(0) / Mc
        assert np.isclose(M[cid], Mc, rtol=1e-14)
        assert np.allclose(Z[cid], Zc, rtol=1e-13, atol=1e-15)
        x = pc - Z[cid]
        assert np.isclose(R[cid], np.linalg.norm(x, axis=1).max(), rtol=1e-15)
        for k, (a, bb, cc) in enumerate(flat):
            ref = (mc * x[:, 0] ** a * x[:, 1] ** bb * x[:, 2] ** cc).sum()
            scl = Mc * max(R[cid], 1e-300) ** (a + bb + cc)
            assert abs(mom[cid, k] - ref) <= 1e-13 * scl + 1e-300
        # dipole about the centre of mass vanishes (Sec. 2) up to the rounding of Z
        assert np.abs(mom[cid, 1:4]).max() <= 1e-13 * Mc * (R[cid] + np.abs(Zc).max())


# ---------------------------------------------------------------------------
# the dual-tree walk (a5) and the opening criterion (a6)
# ---------------------------------------------------------------------------
def _coverage(o):
    """Count how often every unordered body pair is covered by the lists."""
    key, order, _, _ = o.keys()
    c = o.cells()
    m2l, p2p, slf = o.lists()
    n = o.n
    cov = np.zeros((n, n), dtype=np.int64)
    body = lambda cid: np.arange(c.begin[cid], c.begin[cid] + c.count[cid])
    for A, B in np.concatenate([m2l, p2p]):
        ia, ib = body(A), body(B)
        cov[np.ix_(ia, ib)] += 1
        cov[np.ix_(ib, ia)] += 1
    for A in slf:
        ia = body(A)
        cov[np.ix_(ia, ia)] += 1
    np.fill_diagonal(cov, 0)
    return cov


@pytest.mark.parametrize("theta", [0.3, 0.5, 1.0])
def test_walk_covers_every_body_pair_exactly_once(theta):
    b = ics.plummer(700, seed=5)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, theta, 10)
    cov = _coverage(o)
    off = ~np.eye(o.n, dtype=bool)
    assert np.all(cov[off] == 1)


def test_walk_decisions_follow_the_criterion():
    b = ics.plummer(1500, seed=6)
    theta = 0.5
    o = oracle.Oracle(b.x, b.y, b.z, b.m, theta, 25)
    _, Z, R, _ = o.geometry()
    c = o.cells()
    m2l, p2p, slf = o.lists()
    d = np.linalg.norm(Z[m2l[:, 0]] - Z[m2l[:, 1]], axis=1)
    # the paper's form of the criterion, |Z_A - Z_B| >= (R_A + R_B) / theta
    assert np.all(d * (1 + 1e-12) >= (R[m2l[:, 0]] + R[m2l[:, 1]]) / theta)
    dp = np.linalg.norm(Z[p2p[:, 0]] - Z[p2p[:, 1]], axis=1)
    assert np.all(dp * (1 - 1e-12) < (R[p2p[:, 0]] + R[p2p[:, 1]]) / theta)
    assert np.all(c.nchild[p2p.ravel()] == 0) and np.all(c.nchild[slf] == 0)
    assert np.all(m2l[:, 0] < m2l[:, 1]) and np.all(p2p[:, 0] < p2p[:, 1])


# ---------------------------------------------------------------------------
# one accepted pair: force balance (Eq. "unit") and the net torque (Eq. 7/8)
# ---------------------------------------------------------------------------
def _pair_setup(seed=7, n=3000):
    b = ics.plummer(n, seed=seed)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    m2l, _, _ = o.lists()
    c = o.cells()
    # a few accepted pairs with several bodies on both sides
    good = [k for k in range(len(m2l)) if c.count[m2l[k, 0]] >= 4 and c.count[m2l[k, 1]] >= 4]
    return b, o, m2l[good[:: max(1, len(good) // 6)][:6]]


def _octupole(p, m, Zc):
    x = p - Zc
    return np.einsum("n,ni,nj,nk->ijk", m, x, x, x)


def _Dijk(r):
    """Eq. for D_ijk printed in Sec. 2, evaluated at r (test's own copy)."""
    R = np.linalg.norm(r)
    d = np.eye(3)
    return (15 * np.einsum("i,j,k->ijk", r, r, r)
            - 3 * R * R * (np.einsum("ij,k->ijk", d, r) + np.einsum("jk,i->ijk", d, r) +
                           np.einsum("ki,j->ijk", d, r))) / R ** 7


@pytest.mark.parametrize("variant", ["UC", "TC", "TCO"])
def test_pair_force_balance(variant):
    b, o, pairs = _pair_setup()
    for A, B in pairs:
        a = o.pair_accel(A, B, variant)
        f = (b.m[:, None] * a).sum(0)
        assert np.abs(f).max() <= 1e-14 * (b.m[:, None] * np.abs(a)).sum(0).max()


def test_pair_net_torque_closed_form_uc_and_cancelled_tc_tco():
    """UC: the pair's net torque equals 1/2 eps_piq (M_A O_B - O_A M_B)_pjk
    D_ijk(r) (the net torque equation, with r = Z_A - Z_B); TC and TCO: zero
    to rounding."""
    b, o, pairs = _pair_setup()
    p = b.pos()
    M, Z, R, _ = o.geometry()
    eps = np.zeros((3, 3, 3))
    for i, j, k in itertools.permutations(range(3)):
        eps[i, j, k] = np.linalg.det(np.eye(3)[[i, j, k]])
    for A, B in pairs:
        ia, ib = o.cell_bodies(A), o.cell_bodies(B)
        OA = _octupole(p[ia], b.m[ia], Z[A])
        OB = _octupole(p[ib], b.m[ib], Z[B])
        r = Z[A] - Z[B]
        S = M[A] * OB - OA * M[B]
        tau = 0.5 * np.einsum("piq,pjk,ijk->q", eps, S, _Dijk(r))
        scale = {}
        for v in ("UC", "TC", "TCO"):
            a = o.pair_accel(A, B, v)
            t = (b.m[:, None] * np.cross(p, a)).sum(0)
            scale[v] = (b.m[:, None] * np.abs(np.cross(p, a))).sum(0).max()
            if v == "UC":
                assert np.allclose(t, tau, rtol=1e-9, atol=1e-12 * scale[v])
                assert np.linalg.norm(tau) > 1e-9 * scale[v]
            else:
                assert np.abs(t).max() <= 1e-14 * scale[v]


def test_single_body_cells_interact_exactly():
    """Cells of one body each: the expansion is exact (no moments beyond the
    monopole), so the M2L of such a pair equals the direct two-body force."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        p = rng.normal(size=(2, 3))
        m = rng.uniform(0.5, 2.0, 2)
        o = oracle.Oracle(p[:, 0], p[:, 1], p[:, 2], m, 0.5, 1)
        m2l, p2p, slf = o.lists()
        assert len(m2l) == 1 and len(p2p) == 0  # self entries of one-body leaves add nothing
        for v in ("UC", "TC", "TCO"):
            a = o.accel(v)
            ref = oracle.direct(p[:, 0], p[:, 1], p[:, 2], m)
            assert np.allclose(a, ref, rtol=1e-13, atol=0)


# ---------------------------------------------------------------------------
# whole solves: brute force, theta -> 0, balance metric, error ordering
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def plummer2000():
    b = ics.plummer(2000, seed=0)
    ref = oracle.direct(b.x, b.y, b.z, b.m)
    return b, ref


def test_theta_to_zero_reduces_to_direct_summation(plummer2000):
    b, ref = plummer2000
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 1e-7, 25)
    a = o.accel("TC")
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() < 1e-13


def test_force_error_falls_with_theta(plummer2000):
    b, ref = plummer2000
    errs = []
    for theta in (0.3, 0.5, 0.7):
        o = oracle.Oracle(b.x, b.y, b.z, b.m, theta, 25)
        errs.append(oracle.force_errors(o.accel("TC"), ref)["rms"])
    assert errs[0] < errs[1] < errs[2]
    assert errs[1] < 1e-2 and errs[0] < 2e-3


def test_balance_metric_and_paper_orderings(plummer2000):
    """Sec. 3: force balance at machine precision for every variant; torque
    balance at machine precision for TC and TCO, far worse for UC; error
    TC ~ UC and TCO higher."""
    b, ref = plummer2000
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    res = {}
    for v in ("UC", "TC", "TCO"):
        a = o.accel(v)
        res[v] = (oracle.balance(b.x, b.y, b.z, b.m, a), oracle.force_errors(a, ref)["mean"])
    for v in res:
        assert res[v][0][0] < 1e-15
    assert res["TC"][0][1] < 1e-15 and res["TCO"][0][1] < 1e-15
    assert res["UC"][0][1] > 1e3 * res["TC"][0][1]
    assert abs(res["TC"][1] - res["UC"][1]) < 0.2 * res["UC"][1]
    assert res["TCO"][1] > res["TC"][1]


def test_balance_metric_definition():
    x = np.array([1.0, -1.0, 0.0])
    y = np.array([0.0, 0.0, 2.0])
    z = np.zeros(3)
    m = np.array([1.0, 1.0, 2.0])
    a = np.array([[1.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    fb, tb = oracle.balance(x, y, z, m, a)
    assert fb == 0.0
    a2 = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    fb2, _ = oracle.balance(x, y, z, m, a2)
    assert fb2 == 1.0


# ---------------------------------------------------------------------------
# general order P (App. A)
# ---------------------------------------------------------------------------
def test_generic_order3_equals_explicit(plummer2000):
    b, _ = plummer2000
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25, P=3)
    for v in ("UC", "TC", "TCO"):
        g = o.accel(v, generic=True)
        e = o.accel(v)
        if v == "TCO":
            continue
        assert np.abs(g - e).max() <= 1e-13 * np.abs(e).max()


def test_order3_tco_forms_differ_only_along_r():
    """At P = 3 the two D' definitions (Eq. 8 keeps the terms of D_ijkl without
    a factor r_i; App. A projects D onto the plane normal to r) give
    corrective forces that differ only by a component along r."""
    b, o, pairs = _tco_pairs(3)
    M, Z, _, _ = o.geometry()
    for A, B in pairs:
        r = Z[A] - Z[B]
        ia = o.cell_bodies(A)
        d = (o.pair_accel(A, B, "TCO", generic=True) - o.pair_accel(A, B, "TCO"))[ia] * M[A]
        F, _, _ = _pair_corrections(o, A, B)
        scale = np.linalg.norm(F, axis=1).max() * np.linalg.norm(r)
        assert np.abs(np.cross(d, r)).max() <= 1e-10 * scale


@pytest.mark.parametrize("P", [4, 5])
def test_generic_order_torque_cancellation(P):
    b = ics.plummer(600, seed=12)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.6, 16, P=P)
    m2l, _, _ = o.lists()
    p = b.pos()
    c = o.cells()
    sel = [k for k in range(len(m2l)) if c.count[m2l[k, 0]] >= 3 and c.count[m2l[k, 1]] >= 3][:4]
    for k in sel:
        A, B = m2l[k]
        for v in ("UC", "TC", "TCO"):
            a = o.pair_accel(A, B, v, generic=True)
            f = (b.m[:, None] * a).sum(0)
            t = (b.m[:, None] * np.cross(p, a)).sum(0)
            sc = (b.m[:, None] * np.abs(np.cross(p, a))).sum(0).max()
            assert np.abs(f).max() <= 1e-13 * (b.m[:, None] * np.abs(a)).sum(0).max()
            if v == "UC":
                assert np.abs(t).max() > 1e-10 * sc
            else:
                assert np.abs(t).max() <= 1e-13 * sc


def _tco_pairs(P):
    b = ics.plummer(600, seed=12)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.6, 16, P=P)
    m2l, _, _ = o.lists()
    c = o.cells()
    sel = [k for k in range(len(m2l)) if c.count[m2l[k, 0]] >= 3 and c.count[m2l[k, 1]] >= 3][:4]
    return b, o, [tuple(m2l[k]) for k in sel]


def _pair_corrections(o, A, B):
    """(F_c, F'_c, r) of one accepted pair at general order: the corrective
    force is what TC (resp. TCO) adds to UC, times M_A, at every body of A."""
    M, Z, _, _ = o.geometry()
    uc = o.pair_accel(A, B, "UC", generic=True)
    ia = o.cell_bodies(A)
    F = (o.pair_accel(A, B, "TC", generic=True) - uc)[ia] * M[A]
    Fp = (o.pair_accel(A, B, "TCO", generic=True) - uc)[ia] * M[A]
    return F, Fp, Z[A] - Z[B]


@pytest.mark.parametrize("P", [3, 4, 5])
def test_generic_tco_projection_is_perpendicular_to_r(P):
    """App. A's projected D' = (delta - r r / r^2) D makes the TCO corrective
    force the part of F_c perpendicular to r: r . F'_c = 0 and F_c - F'_c is
    parallel to r, the same force on every body of A.  (A flipped projection
    F_c + r (r.F_c)/r^2 still cancels the torque and balances the force, so
    only this pin sees it.)"""
    _, o, pairs = _tco_pairs(P)
    for A, B in pairs:
        F, Fp, r = _pair_corrections(o, A, B)
        scale = np.linalg.norm(F, axis=1).max() * np.linalg.norm(r)
        assert np.abs(Fp @ r).max() <= 1e-10 * scale
        assert np.abs(F - F[0]).max() <= 1e-10 * np.abs(F).max()
        par = np.cross(F - Fp, r)
        assert np.abs(par).max() <= 1e-10 * scale
        # the projection removes a component that is really there
        assert np.abs(F @ r).max() > 1e-3 * scale


def test_higher_order_is_more_accurate():
    b = ics.plummer(800, seed=13)
    ref = oracle.direct(b.x, b.y, b.z, b.m)
    e = {}
    for P in (3, 4, 5):
        o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.6, 16, P=P)
        e[P] = oracle.force_errors(o.accel("TC", generic=True), ref)["rms"]
    assert e[5] < e[4] < e[3]


# ---------------------------------------------------------------------------
# planted mistakes: the pins above must catch them (run on the CPU)
# ---------------------------------------------------------------------------
def test_planted_half_coefficient_breaks_torque_pin():
    """Eq. (7) as printed (coefficient 1/2 instead of App. A's 1/6) would
    leave a residual torque of -2 tau: the closed-form pin would fail."""
    b, o, pairs = _pair_setup()
    p = b.pos()
    A, B = pairs[0]
    a_uc = o.pair_accel(A, B, "UC")
    a_tc = o.pair_accel(A, B, "TC")
    corr = a_tc - a_uc  # the correction F/M_A, -F/M_B at each body
    wrong = a_uc + 3.0 * corr
    t = (b.m[:, None] * np.cross(p, wrong)).sum(0)
    t_uc = (b.m[:, None] * np.cross(p, a_uc)).sum(0)
    assert np.allclose(t, -2.0 * t_uc, rtol=1e-6)
    sc = (b.m[:, None] * np.abs(np.cross(p, wrong))).sum(0).max()
    assert np.abs(t).max() > 1e-10 * sc


@pytest.mark.parametrize("P", [4, 5])
def test_planted_projection_sign_flip_breaks_perpendicular_pin(P):
    """A TCO projection with the wrong sign, F_c + r (r.F_c)/r^2, cancels the
    torque like the right one (it differs by a force along r) but leaves
    r . F'_c = 2 r . F_c: the perpendicularity pin above fails on it."""
    b, o, pairs = _tco_pairs(P)
    p = b.pos()
    M, _, _, _ = o.geometry()
    for A, B in pairs[:2]:
        F, _, r = _pair_corrections(o, A, B)
        flipped = F + np.outer(F @ r, r) / (r @ r)
        scale = np.linalg.norm(F, axis=1).max() * np.linalg.norm(r)
        assert np.abs(flipped @ r).max() > 1e-6 * scale
        # ... while the torque pin alone cannot tell: the flipped force, put
        # back into the pair's accelerations, still cancels the torque
        uc = o.pair_accel(A, B, "UC", generic=True)
        a = uc.copy()
        ia, ib = o.cell_bodies(A), o.cell_bodies(B)
        a[ia] += flipped[0] / M[A]
        a[ib] -= flipped[0] / M[B]
        t = (b.m[:, None] * np.cross(p, a)).sum(0)
        sc = (b.m[:, None] * np.abs(np.cross(p, a))).sum(0).max()
        assert np.abs(t).max() <= 1e-12 * sc


def test_planted_sign_flip_breaks_brute_force_pin(plummer2000):
    """Evaluating the expansion at R = Z_B - Z_A (the paper's Sec. 2
    definition) flips every odd derivative; the far field then points the
    wrong way and the brute-force pin fails."""
    b, ref = plummer2000
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    far = o.accel("TC", parts=oracle.PART_FAR)
    near = o.accel("TC", parts=oracle.PART_NEAR)
    ok = oracle.force_errors(far + near, ref)["rms"]
    bad = oracle.force_errors(near - far, ref)["rms"]
    assert ok < 1e-2 < bad
