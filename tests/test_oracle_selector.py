"""Pins of the selector's oracle parts (CPU): the Adam step of the training,
the walk with the learned selector (oracle/selector_walk.py), its pair
features and field estimate, and the oracle's evaluation of caller-given
interaction lists."""
import numpy as np
import pytest

import oracle
from oracle import mlp as M
from oracle import selector_walk as SW
from paper_1706_06989_gb300 import ics


# ---------------------------------------------------------------------------
# Adam (Kingma & Ba 2015, Algorithm 1)
# ---------------------------------------------------------------------------
def test_adam_first_step_moves_each_weight_by_lr_times_sign():
    """With zero moments, the bias-corrected first step is
    lr * g / (|g| + eps): lr * sign(g) up to eps, whatever |g| is."""
    rng = np.random.default_rng(0)
    p = rng.normal(size=M.NPARAMS)
    g = rng.normal(size=M.NW) * 10.0 ** rng.uniform(-4, 2, M.NW)
    g[5] = 0.0
    z = np.zeros(M.NW)
    p1, m1, v1 = M.adam_step(p, z, z, g, lr=1e-2, step=1)
    expect = p[:M.NW] - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p1[:M.NW], expect, rtol=0, atol=1e-15)
    assert p1[5] == p[5]  # a zero gradient moves nothing
    assert np.array_equal(p1[M.NW:], p[M.NW:])  # normalisation untouched
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_hand_computed_second_step():
    """Two steps with gradients 3 and then -1 on one weight (beta 0.9 /
    0.999, eps 1e-8, lr 0.1), worked by hand:
      m1 = 0.3,            v1 = 0.009,
      m2 = 0.27 - 0.1 = 0.17,          v2 = 0.008991 + 0.001 = 0.009991,
      m2_hat = 0.17 / 0.19 = 0.894736842...,  v2_hat = 0.009991 / 0.001999,
      step 2 = -0.1 * m2_hat / (sqrt(v2_hat) + 1e-8)."""
    p = np.zeros(M.NPARAMS)
    z = np.zeros(M.NW)
    g1 = np.zeros(M.NW)
    g1[0] = 3.0
    g2 = np.zeros(M.NW)
    g2[0] = -1.0
    p1, m1, v1 = M.adam_step(p, z, z, g1, lr=0.1, step=1)
    assert abs(p1[0] - (-0.1 * 3.0 / (3.0 + 1e-8))) < 1e-15
    p2, m2, v2 = M.adam_step(p1, m1, v1, g2, lr=0.1, step=2)
    assert abs(m2[0] - 0.17) < 1e-15 and abs(v2[0] - 0.009991) < 1e-15
    step2 = -0.1 * (0.17 / 0.19) / (np.sqrt(0.009991 / 0.001999) + 1e-8)
    assert abs((p2[0] - p1[0]) - step2) < 1e-14
    assert abs(step2 - (-0.040021)) < 1e-6  # the worked value, to six places


def test_adam_constant_gradient_keeps_unit_steps():
    """A constant gradient gives m_hat = g and v_hat = g^2 at every step
    (the bias correction undoes the zero start), so every step is lr."""
    p = np.zeros(M.NPARAMS)
    m = v = np.zeros(M.NW)
    g = np.full(M.NW, 0.37)
    for t in range(1, 6):
        q, m, v = M.adam_step(p, m, v, g, lr=0.01, step=t)
        assert np.allclose(q[:M.NW] - p[:M.NW], -0.01, rtol=1e-7)
        p = q


# ---------------------------------------------------------------------------
# selector walk
# ---------------------------------------------------------------------------
def _params(seed=0):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=M.NPARAMS) * 0.15).astype(np.float32)
    p[M.NW:M.NW + 8] = rng.normal(size=8).astype(np.float32)
    p[M.NW + 8:] = rng.uniform(0.5, 1.5, 8).astype(np.float32)
    return p


def _const_net(b4):
    p = _params(3)
    p[M.NW - 65:M.NW - 1] = 0.0  # w4 = 0: the output is b4
    p[M.NW - 1] = b4
    return p


@pytest.fixture(scope="module")
def plummer3000():
    b = ics.plummer(3000, seed=9)
    return b, {th: oracle.Oracle(b.x, b.y, b.z, b.m, th, 25) for th in (0.5, 0.7, 1.0)}


@pytest.mark.parametrize("rule", [SW.ABSOLUTE, SW.RELATIVE])
def test_selector_walk_extremes_equal_the_plain_walk(plummer3000, rule):
    """theta is a floor and theta_max a ceiling: a network that rejects every
    pair leaves the C oracle's walk at theta; one that accepts every band
    pair gives the C oracle's walk at theta_max."""
    b, o = plummer3000
    for b4, th_max, th in ((100.0, 1.0, 0.5), (-100.0, 1.0, 1.0), (-100.0, 0.7, 0.7)):
        got = SW.canonical(*SW.walk(o[0.5], _const_net(b4), -3.0, th_max, 0, rule)[:3])
        ref = SW.canonical(*o[th].lists())
        for g, r in zip(got, ref):
            assert np.array_equal(g, r), (b4, th_max, th)


def _coverage(o, m2l, p2p, slf, n):
    order = o.keys()[1]
    c = o.cells()
    body = lambda cid: order[c.begin[cid]:c.begin[cid] + c.count[cid]]
    cov = np.zeros((n, n), dtype=np.int32)
    for A, B in np.concatenate([m2l.reshape(-1, 2), p2p.reshape(-1, 2)]):
        ia, ib = body(A), body(B)
        cov[np.ix_(ia, ib)] += 1
        cov[np.ix_(ib, ia)] += 1
    for A in slf:
        ia = body(A)
        cov[np.ix_(ia, ia)] += 1
    np.fill_diagonal(cov, 1)
    return np.all(cov == 1)


@pytest.mark.parametrize("rule", [SW.ABSOLUTE, SW.RELATIVE])
def test_selector_walk_is_complete_safe_and_between_the_bounds(plummer3000, rule):
    """With a random network at a target that accepts part of the band: every
    body pair is covered exactly once, every accepted pair meets the safety
    bound |Z_A - Z_B| >= R_A + R_B, and the M2L count lies between those of
    the plain walks at theta and theta_max."""
    b, o = plummer3000
    p = _params(2)
    _, _, _, sc = SW.walk(o[0.5], p, 0.0, 1.0, 64, rule)
    tgt = float(np.median(list(sc.values())))
    m2l, p2p, slf, sc = SW.walk(o[0.5], p, tgt, 1.0, 64, rule)
    acc = sum(1 for v in sc.values() if v < tgt)
    assert 0 < acc < len(sc)
    assert _coverage(o[0.5], m2l, p2p, slf, b.n)
    _, Z, R, _ = o[0.5].geometry()
    d = np.linalg.norm(Z[m2l[:, 0]] - Z[m2l[:, 1]], axis=1)
    assert np.all(d * (1 + 1e-12) >= R[m2l[:, 0]] + R[m2l[:, 1]])
    # every scored pair that was accepted appears in the M2L list
    mset = set(map(tuple, m2l.tolist()))
    assert all((k in mset) == (v < tgt) for k, v in sc.items())


def test_pair_features_by_definition(plummer3000):
    """The eight features of sampled pairs, recomputed from the bodies of the
    two cells: centre of mass, R_max as the largest body distance, and the
    trace-free quadrupole from the bodies' offsets."""
    b, o = plummer3000
    oo = o[0.5]
    m2l, _, _ = oo.lists()
    sel = m2l[:: max(1, len(m2l) // 60)]
    f, ordered = SW.pair_features(oo, sel)
    p = b.pos()
    _, _, R, _ = oo.geometry()
    for k, (A, B) in enumerate(sel):
        a_, b_ = ordered[k]
        assert {a_, b_} == {A, B}
        assert np.float32(R[a_]) > np.float32(R[b_]) or (np.float32(R[a_]) == np.float32(R[b_]) and a_ < b_)
        props = []
        for c in (a_, b_):
            ii = oo.cell_bodies(c)
            mc = b.m[ii].sum()
            zc = (b.m[ii, None] * p[ii]).sum(0) / mc
            x = p[ii] - zc
            rmax = np.linalg.norm(x, axis=1).max()
            Q = np.einsum("n,ni,nj->ij", b.m[ii], x, x)
            Qt = Q - np.trace(Q) / 3 * np.eye(3)
            qn = np.linalg.norm(Qt) / (mc * rmax ** 2) if (rmax > 0 and len(ii) > 1) else 0.0
            props.append((mc, zc, rmax, qn, len(ii)))
        (ma, za, ra, qa, na), (mb, zb, rb, qb, nb) = props
        r = np.linalg.norm(za - zb)
        ref = [np.log10(r), max(np.log10(ra / r) if ra > 0 else -np.inf, -12), max(np.log10(rb / r) if rb > 0 else -np.inf, -12),
               np.log10(ma), np.log10(mb), np.log10(qa + 1e-12), np.log10(qb + 1e-12), np.log10(na + nb)]
        assert np.allclose(f[k], ref, rtol=0, atol=1e-9), (k, f[k], ref)


def test_field_estimate_of_separated_clusters():
    """Three compact clusters of unequal mass in three octants of the root:
    each is one leaf at level 1, the coarse level.  The estimate at a
    cluster's centre is the softened monopole field of the other two, which
    for clusters this small is the exact field there to about 1e-4 (a wrong
    power, mass factor or sign is far off)."""
    rng = np.random.default_rng(5)
    centres = np.array([[-10.0, -10.0, -10.0], [10.0, -10.0, 10.0], [-10.0, 10.0, 10.0]])
    masses = np.array([1.0, 2.5, 0.7])
    p, m = [], []
    for c, mc in zip(centres, masses):
        p.append(c + 0.01 * rng.normal(size=(6, 3)))
        m.append(np.full(6, mc / 6))
    p, m = np.concatenate(p), np.concatenate(m)
    o = oracle.Oracle(p[:, 0], p[:, 1], p[:, 2], m, 0.5, 8)
    lev = o.cells().level
    assert lev.max() == 1 and (lev == 1).sum() == 3
    lga = SW.field_estimate(o)
    _, Z, _, _ = o.geometry()
    for c in np.nonzero(lev == 1)[0]:
        own = np.linalg.norm(p - Z[c], axis=1) < 1.0
        d = p[~own] - Z[c]
        r = np.linalg.norm(d, axis=1)
        exact = np.linalg.norm(((m[~own] / r ** 3)[:, None] * d).sum(0))
        assert abs(10.0 ** lga[c] / exact - 1.0) < 1e-3


def test_set_lists_evaluates_another_selection():
    """Giving a theta = 0.5 tree the lists of the theta = 1 walk reproduces the
    theta = 1 oracle's forces exactly (same tree, same pairs); its own lists
    reproduce its own forces; a P2P entry that is not a leaf is refused."""
    b = ics.plummer(1500, seed=4)
    o5 = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    o1 = oracle.Oracle(b.x, b.y, b.z, b.m, 1.0, 25)
    a5 = o5.accel("TC")
    a1 = o1.accel("TC")
    lists1 = o1.lists()
    o5.set_lists(*o5.lists())
    assert np.array_equal(o5.accel("TC"), a5)
    o5.set_lists(*lists1)
    assert np.abs(o5.accel("TC") - a1).max() <= 1e-14 * np.abs(a1).max()
    with pytest.raises(oracle.OracleError):
        o5.set_lists(np.zeros((0, 2)), np.array([[0, 1]]), np.zeros(0))
