"""a12: the learned pair selector on the GPU -- network forward and gradient
against the reference network, features and labels against the oracle, and
the walk with the selector (mutual pairs, conservation, coverage)."""
import numpy as np
import pytest

import oracle
from oracle import mlp as M
from oracle import selector_walk as SW
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(**kw):
    from paper_1706_06989_gb300 import fmm
    return fmm.FMM(**kw)


def _dev(b):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))


def _params(seed=0):
    rng = np.random.default_rng(seed)
    p = (rng.normal(size=M.NPARAMS) * 0.15).astype(np.float32)
    p[M.NW:M.NW + 8] = rng.normal(size=8).astype(np.float32)
    p[M.NW + 8:] = rng.uniform(0.5, 1.5, 8).astype(np.float32)
    return p


def test_mlp_forward_and_gradient_match_reference():
    s = _solver()
    rng = np.random.default_rng(4)
    p = _params(1)
    X = rng.normal(size=(1000, 8)).astype(np.float32) * 2
    y = rng.normal(size=1000).astype(np.float32)
    pd = torch.from_numpy(p).cuda()
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    out = s.mlp_forward(pd, Xd).cpu().numpy()
    ref, _, _ = M.forward(p, X, "bf16")
    assert np.abs(out - ref).max() <= 2e-3 * (1 + np.abs(ref).max())
    g, loss = s.mlp_grad(pd, Xd, yd)
    rl, rg = M.loss_and_grad(p, X, y, "bf16")
    g = g.cpu().numpy()[:M.NW]
    assert abs(float(loss.cpu()) - rl) <= 1e-3 * rl
    # entry by entry, per tensor: the two sides round the same operands to
    # BF16 at the same places but sum the FP32 products in different orders,
    # so an entry may differ by a few BF16 roundings of its own terms; the
    # bound scales with the entry and with the tensor's largest entry
    _compare_gradient(g, rg)
    g2, _ = s.mlp_grad(pd, Xd, yd)
    assert np.array_equal(g, g2.cpu().numpy()[:M.NW])  # reproducible


_TENSORS = (("W1", 64 * 8), ("b1", 64), ("W2", 64 * 64), ("b2", 64), ("W3", 64 * 64), ("b3", 64), ("w4", 64),
            ("b4", 1))


def _compare_gradient(g, rg):
    o = 0
    for name, n in _TENSORS:
        a, r = g[o:o + n], rg[o:o + n]
        o += n
        bound = 2e-2 * np.abs(r) + 2e-3 * np.abs(r).max()
        bad = np.abs(a - r) > bound
        assert not bad.any(), (name, int(bad.sum()), float(np.abs(a - r).max()), float(np.abs(r).max()))
        # a flipped sign or a dropped factor on a whole tensor shows in its norm
        assert np.linalg.norm(a - r) <= 1e-2 * np.linalg.norm(r), name
    assert o == M.NW


def test_mlp_gradient_entrywise_at_training_scale():
    """The gradient of a batch of the size the training uses, on trained-like
    inputs (features spread like the method's, labels in the label range)."""
    s = _solver()
    rng = np.random.default_rng(11)
    p = _params(5)
    X = (rng.normal(size=(8192, 8)) * np.array([0.5, 0.4, 0.4, 1.0, 1.0, 0.5, 0.5, 0.8]) +
         np.array([-1.0, -0.5, -0.7, -5.0, -5.0, -1.0, -1.0, 1.5])).astype(np.float32)
    y = rng.uniform(-6, -1, 8192).astype(np.float32)
    pd = torch.from_numpy(p).cuda()
    g, loss = s.mlp_grad(pd, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    rl, rg = M.loss_and_grad(p, X, y, "bf16")
    assert abs(float(loss.cpu()) - rl) <= 1e-3 * rl
    _compare_gradient(g.cpu().numpy()[:M.NW], rg)


def test_adam_step_matches_oracle():
    """One Adam step of the device optimiser against the oracle's Adam
    (Kingma & Ba 2015), element by element: FP32 on the device, FP64 in the
    oracle, from the same parameters, moments and gradient."""
    s = _solver()
    rng = np.random.default_rng(12)
    p = _params(6)
    m0 = (rng.normal(size=M.NW) * 1e-2).astype(np.float32)
    v0 = (rng.uniform(0, 1e-3, M.NW)).astype(np.float32)
    g = (rng.normal(size=M.NW) * 10.0 ** rng.uniform(-5, 0, M.NW)).astype(np.float32)
    for step in (1, 7):
        pd = torch.from_numpy(p.copy()).cuda()
        md = torch.from_numpy(m0.copy()).cuda()
        vd = torch.from_numpy(v0.copy()).cuda()
        gd = torch.from_numpy(g).cuda()
        import ctypes
        rc = s.lib.fmm_mlp_adam(s._h, ctypes.c_void_p(pd.data_ptr()), ctypes.c_void_p(md.data_ptr()),
                                ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(gd.data_ptr()), 3e-3, step)
        assert rc == 0
        # the device holds beta1, beta2, eps and lr as FP32 constants: the
        # oracle takes those same values (1 - float32(0.999) differs from
        # 0.001 by 1.3e-5 of itself)
        f32 = lambda v: float(np.float32(v))
        rp, rm, rv = M.adam_step(p.astype(np.float64), m0, v0, g, f32(3e-3), step, beta1=f32(0.9),
                                 beta2=f32(0.999), eps=f32(1e-8))
        gp, gm, gv = pd.cpu().numpy(), md.cpu().numpy(), vd.cpu().numpy()
        # FP32 rounding relative to the size of the terms (the two terms of a
        # moment can cancel, so the bound follows the terms, not the result)
        tm = 0.9 * np.abs(m0) + 0.1 * np.abs(g)
        tv = 0.999 * np.abs(v0) + 0.001 * g.astype(np.float64) ** 2
        assert np.all(np.abs(gm - rm) <= 4e-7 * tm)
        assert np.all(np.abs(gv - rv) <= 4e-7 * tv)
        # the move: lr m_hat / (sqrt(v_hat) + eps) with the same relative
        # rounding in m_hat, plus the FP32 rounding of p itself
        mv, rmv = gp[:M.NW].astype(np.float64) - p[:M.NW], rp[:M.NW] - p[:M.NW]
        vh = rv / (1 - 0.999 ** step)
        bound = 1e-5 * 3e-3 * (tm / (1 - 0.9 ** step)) / (np.sqrt(vh) + 1e-8) + 2e-5 * np.abs(rmv)
        assert np.all(np.abs(mv - rmv) <= bound + np.spacing(np.abs(p[:M.NW]).astype(np.float32)))
        assert np.array_equal(gp[M.NW:], p[M.NW:])


def test_features_and_labels_match_oracle():
    b = ics.plummer(3000, seed=5)
    s = _solver(theta=0.5)
    x, y, z, m = _dev(b)
    s.solve(x, y, z, m)
    m2l, _, _ = s.export_lists()
    sel = m2l[::max(1, m2l.shape[0] // 150)].contiguous()
    feat, lab = s.selector_samples(sel)
    feat, lab, sel = feat.cpu().numpy(), lab.cpu().numpy(), sel.cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    Mc, Zc, R, mom = o.geometry()
    cnt = o.cells().count
    p = b.pos()
    ofeat, _ = SW.pair_features(o, sel)
    for k, (A, B) in enumerate(sel):
        ra, rb = np.float32(R[A]), np.float32(R[B])  # pairs are ordered by R_max in FP32
        if rb > ra or (rb == ra and B < A):
            A, B = B, A
        r = np.linalg.norm(Zc[A] - Zc[B])
        assert abs(feat[k, 0] - np.log10(r)) < 1e-5
        assert abs(feat[k, 1] - np.log10(max(R[A] / r, 1e-12))) < 1e-5
        assert abs(feat[k, 7] - np.log10(cnt[A] + cnt[B])) < 1e-5
        # all eight against the oracle's features of the same pair
        assert np.abs(feat[k] - ofeat[k]).max() < 2e-5, (k, feat[k], ofeat[k])
        # label: the worse side's rms |a_M2L - a_direct| for this pair alone,
        # relative to the other cell's monopole field
        a = o.pair_accel(A, B, "TC")
        ia, ib = o.cell_bodies(A), o.cell_bodies(B)
        dire = np.zeros_like(a)
        for tgt, src in ((ia, ib), (ib, ia)):
            d = p[src][None, :, :] - p[tgt][:, None, :]
            rr = np.linalg.norm(d, axis=2)
            dire[tgt] = np.einsum("ijk,j->ik", d / rr[:, :, None] ** 3, b.m[src])
        def side(ii, m_other):
            if ii.size > 128:  # 128 evenly spaced targets stand for a big side
                ii = ii[(np.arange(128) * ii.size) // 128]
            return np.sqrt(np.mean(np.sum((a[ii] - dire[ii]) ** 2, axis=1))) / (m_other / r ** 2)
        ref = max(np.log10(max(side(ia, Mc[B]), side(ib, Mc[A])) + 1e-300), -12.0)
        if ref < -11.0:  # rounding-level errors: both at the floor region
            assert lab[k] < -10.5, (k, lab[k], ref)
        else:
            assert abs(lab[k] - ref) < 1e-4, (k, lab[k], ref)


def _coverage_ok(s, n):
    c = s.export_tree(geometry=False)
    begin, count = c["begin"].cpu().numpy(), c["count"].cpu().numpy()
    _, order = s.export_keys()
    order = order.cpu().numpy()
    m2l, p2p, slf = (t.cpu().numpy() for t in s.export_lists())
    cov = np.zeros((n, n), dtype=np.int32)
    body = lambda cid: order[begin[cid]:begin[cid] + count[cid]]
    for A, B in np.concatenate([m2l, p2p]):
        ia, ib = body(A), body(B)
        cov[np.ix_(ia, ib)] += 1
        cov[np.ix_(ib, ia)] += 1
    for A in slf:
        ia = body(A)
        cov[np.ix_(ia, ia)] += 1
    np.fill_diagonal(cov, 1)
    return np.all(cov == 1)


def test_selector_walk_is_mutual_conserving_and_complete():
    b = ics.plummer(1500, seed=7)
    s = _solver(theta=0.5, variant="TC")
    s.selector_set(_params(2), log10_target=-2.0, enable=True)
    x, y, z, m = _dev(b)
    a = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    assert _coverage_ok(s, b.n)
    _, Zc, R, _ = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25).geometry()
    m2l, _, _ = s.export_lists()
    m2l = m2l.cpu().numpy()
    d = np.linalg.norm(Zc[m2l[:, 0]] - Zc[m2l[:, 1]], axis=1)
    assert np.all(d * (1 + 1e-12) >= R[m2l[:, 0]] + R[m2l[:, 1]])  # safety bound
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, a)
    assert fb <= 1e-13 and tb <= 1e-13
    a2 = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    assert np.array_equal(a, a2)


def test_training_reduces_the_loss():
    from paper_1706_06989_gb300 import selector
    b = ics.plummer(20000, seed=8)
    s = _solver(theta=0.5)
    x, y, z, m = _dev(b)
    feat, lab = selector.pair_samples(s, x, y, z, m, thetas=(0.4, 0.7, 1.0), per_theta=20000, seed=1)
    params, losses = selector.train(s, feat, lab, steps=600, batch=2048, lr=3e-3, seed=2)
    assert losses[-50:].mean() < 0.5 * losses[:20].mean()
    assert np.isfinite(params).all()


def test_selector_extremes_reduce_to_the_plain_criterion():
    """theta is a floor and theta_max a ceiling: a network that accepts nothing
    leaves the walk of the plain criterion at theta; one that accepts every
    pair of the band gives the walk of the criterion at theta_max."""
    b = ics.plummer(3000, seed=9)
    x, y, z, m = _dev(b)
    lists = {}
    for th in (0.5, 0.7, 1.0):
        s = _solver(theta=th)
        s.solve(x, y, z, m)
        lists[th] = [t.cpu().numpy() for t in s.export_lists()]
    p = _params(3)
    p[M.NW - 65:M.NW - 1] = 0.0  # w4: constant output b4
    for b4, th_max, th in ((100.0, 1.0, 0.5), (-100.0, 1.0, 1.0), (-100.0, 0.7, 0.7)):
        p[M.NW - 1] = b4
        s = _solver(theta=0.5)
        s.selector_set(p, log10_target=-3.0, enable=True, theta_max=th_max, min_work=0)
        s.solve(x, y, z, m)
        got = [t.cpu().numpy() for t in s.export_lists()]
        for g, r in zip(got, lists[th]):
            assert np.array_equal(g, r), (b4, th_max, th)
    with pytest.raises(Exception):
        s.selector_set(p, log10_target=-3.0, enable=True, theta_max=1.5)
    # an unknown acceptance rule is refused at the C boundary
    import ctypes
    from paper_1706_06989_gb300 import fmm
    rc = s.lib.fmm_selector_set(s._h, ctypes.c_void_p(p.ctypes.data), -3.0, 1.0, 0, 7, 1)
    assert rc == fmm.FMM_EINVAL


def _gpu_lists(s):
    return SW.canonical(*(t.cpu().numpy() for t in s.export_lists()))


@pytest.mark.parametrize("rule", ["absolute", "relative"])
def test_selector_lists_match_oracle_selector_walk(rule):
    """The walk with the learned selector against the oracle's selector walk
    (same tree, same network): the lists must be identical, except that a
    pair whose oracle score lies within delta = 1e-2 (log10 units) of the
    target may be decided either way -- the two sides compute the features
    and the network in different orders and precisions.  For those pairs the
    oracle takes the GPU's decision, and the walks must then agree exactly.
    Then the forces of the selected lists are judged by the oracle."""
    b = ics.plummer(4000, seed=21)
    x, y, z, m = _dev(b)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    p = _params(2)
    code = SW.RELATIVE if rule == "relative" else SW.ABSOLUTE
    _, _, _, sc = SW.walk(o, p, 0.0, 1.0, 64, code)
    tgt = float(np.median(list(sc.values())))
    s = _solver(theta=0.5, variant="TC")
    s.selector_set(p, log10_target=tgt, enable=True, theta_max=1.0, min_work=64, rule=rule)
    a = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    gm2l, gp2p, gslf = _gpu_lists(s)
    gset = set(map(tuple, gm2l.tolist()))
    delta = 1e-2
    amb = []

    def decide(A, B, score):
        if abs(score - tgt) <= delta:
            amb.append((A, B))
            return (min(A, B), max(A, B)) in gset
        return score < tgt

    om2l, op2p, oslf, sc = SW.walk(o, p, tgt, 1.0, 64, code, decide=decide)
    om2l, op2p, oslf = SW.canonical(om2l, op2p, oslf)
    assert len(sc) > 50
    assert len(amb) <= 0.05 * len(sc), (len(amb), len(sc))
    assert np.array_equal(gm2l, om2l) and np.array_equal(gp2p, op2p) and np.array_equal(gslf, oslf)
    # a selection that really differs from the plain walk at theta
    plain = SW.canonical(*o.lists())
    assert gm2l.shape[0] != plain[0].shape[0]
    # forces of these lists by the oracle, 1e-12 per body
    o.set_lists(om2l, op2p, oslf)
    ref = o.accel("TC")
    rel = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-12, rel.max()
