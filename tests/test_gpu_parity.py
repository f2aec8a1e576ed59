"""CUDA path against the CPU oracle, through the C ABI (needs a GB300).

Bit-exact: Morton keys, sort order, tree topology, M, Z, R_max (the opening
criterion consumes them) and the interaction lists after a canonical sort.
FP64 accelerations: within 1e-12 relative per body.  Conservation: net force
and torque balance (Sec. 3 metric) at rounding level for TC / TCO.
"""
import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(b):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))


def _solver(**kw):
    from paper_1706_06989_gb300 import fmm
    return fmm.FMM(**kw)


def _solve(b, theta=0.5, n_crit=25, variant="TC", precision="fp64"):
    s = _solver(theta=theta, n_crit=n_crit, variant=variant, precision=precision)
    x, y, z, m = _dev(b)
    ax, ay, az = s.solve(x, y, z, m)
    torch.cuda.synchronize()
    return s, torch.stack([ax, ay, az], 1).cpu().numpy()


def _canon_pairs(p):
    p = np.asarray(p, dtype=np.int64).reshape(-1, 2)
    lo, hi = np.minimum(p[:, 0], p[:, 1]), np.maximum(p[:, 0], p[:, 1])
    k = lo * (1 << 32) + hi
    return np.sort(k)


def _rel_dev(got, ref):
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def _compare_tree(s, o):
    st = s.stats()
    assert st.ncell == o.ncell
    key, order = s.export_keys()
    okey, oorder, lo, scale = o.keys()
    assert np.array_equal(key.cpu().numpy().view(np.uint64), okey)
    assert np.array_equal(order.cpu().numpy(), oorder)
    assert np.array_equal(np.array(st.lo), lo) and st.scale == scale
    t = s.export_tree()
    oc = o.cells()
    for name in ("begin", "count", "level", "parent", "first_child", "nchild"):
        assert np.array_equal(t[name].cpu().numpy(), getattr(oc, name)), name
    M, Z, R, mom = o.geometry()
    # bit-exact: compare the IEEE bit patterns
    assert np.array_equal(t["M"].cpu().numpy().view(np.int64), M.view(np.int64))
    assert np.array_equal(t["Z"].cpu().numpy().view(np.int64), Z.view(np.int64))
    assert np.array_equal(t["Rmax"].cpu().numpy().view(np.int64), R.view(np.int64))
    return mom


def _compare_lists(s, o):
    m2l, p2p, slf = s.export_lists()
    om2l, op2p, oslf = o.lists()
    assert np.array_equal(_canon_pairs(m2l.cpu().numpy()), _canon_pairs(om2l))
    assert np.array_equal(_canon_pairs(p2p.cpu().numpy()), _canon_pairs(op2p))
    assert np.array_equal(np.sort(slf.cpu().numpy()), np.sort(oslf))


@pytest.mark.parametrize("variant", ["UC", "TC", "TCO"])
def test_plummer_2000_matches_oracle(variant):
    b = ics.plummer(2000, seed=0)
    s, got = _solve(b, variant=variant)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_tree(s, o)
    _compare_lists(s, o)
    ref = o.accel(variant)
    rel = _rel_dev(got, ref)
    assert rel.max() <= 1e-12, rel.max()
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert fb <= 1e-13
    if variant != "UC":
        assert tb <= 1e-13


@pytest.mark.parametrize("k,variant", [(-90, "TC"), (90, "TC"), (-90, "UC"), (90, "TCO")])
def test_fp64_far_from_unit_scale(k, variant):
    """Positions scaled by 2^k (masses unchanged): the FP64 path keeps its
    1e-12 parity against the oracle, which takes the same scaled inputs.
    Morton keys, tree and lists are unchanged by a power-of-two scale, and
    the pair factor r^-3 of the near field builds its seed from the
    exponent of r^2 (here near 2^(2k)), so both signs of a large exponent
    are exercised.  (The oracle is exactly covariant at this scale; at
    2^+-120 intermediate powers of R in the oracle leave the FP64 range.)"""
    b0 = ics.plummer(2000, seed=9)
    f = np.ldexp(1.0, k)
    b = ics.Bodies(b0.x * f, b0.y * f, b0.z * f, b0.m)
    s, got = _solve(b, variant=variant)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_lists(s, o)
    rel = _rel_dev(got, o.accel(variant))
    assert rel.max() <= 1e-12, rel.max()
    # the same lists as the unscaled system, and accelerations 2^(-2k) times its own
    s0, got0 = _solve(b0, variant=variant)
    assert s0.stats().n_m2l == s.stats().n_m2l and s0.stats().p2p_body_pairs == s.stats().p2p_body_pairs
    rel0 = _rel_dev(np.ldexp(got, 2 * k), got0)
    assert rel0.max() <= 1e-13, rel0.max()


@pytest.mark.parametrize("k", [-10, 10])
def test_mixed_away_from_unit_scale(k):
    """The mixed form on a Plummer sphere scaled by 2^k (masses unchanged):
    its FP32 terms stay well inside the FP32 range, the lists (decided in
    FP64, with the FP32 filter in front) stay bit-exact, and the rms force
    deviation from the oracle stays within the mixed form's bound."""
    b0 = ics.plummer(2000, seed=10)
    f = np.ldexp(1.0, k)
    b = ics.Bodies(b0.x * f, b0.y * f, b0.z * f, b0.m)
    s, got = _solve(b, precision="mixed")
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_lists(s, o)
    dev = _rel_dev(got, o.accel("TC"))
    assert np.sqrt(np.mean(dev ** 2)) <= 1e-6


def test_moments_match_definition():
    b = ics.plummer(2000, seed=3)
    s, _ = _solve(b)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _, _, R, omom = o.geometry()
    mom = s.export_moments().cpu().numpy()
    M = mom[:, 0]
    # the oracle's multi-index order for orders 0..3 equals the library layout
    for n_ord, sl in ((1, slice(1, 4)), (2, slice(4, 10)), (3, slice(10, 20))):
        ref = omom[:, sl]
        tol = 1e-12 * (M * np.maximum(R, 1e-300) ** n_ord)[:, None] + 1e-300
        assert np.all(np.abs(mom[:, sl] - ref) <= tol), n_ord


def test_uniform_masses_spread_65536():
    b = ics.uniform_cube(65536, seed=5, mass_spread=True)
    s, got = _solve(b, theta=0.6, variant="TC")
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.6, 25)
    _compare_tree(s, o)
    _compare_lists(s, o)
    t = ics.error_subset(b.n, 2048, seed=7)
    ref = o.accel("TC", targets=t)
    assert _rel_dev(got[t], ref).max() <= 1e-12


def test_deterministic_bits():
    b = ics.plummer(30000, seed=2)
    s = _solver(theta=0.5, n_crit=25, variant="TC")
    x, y, z, m = _dev(b)
    a1 = torch.stack(s.solve(x, y, z, m), 1).clone()
    a2 = torch.stack(s.solve(x, y, z, m), 1).clone()
    assert torch.equal(a1.view(torch.int64), a2.view(torch.int64))


def test_host_entry_point_matches_device():
    b = ics.plummer(5000, seed=4)
    s, got = _solve(b)
    hx = s.solve_host(b.x, b.y, b.z, b.m)
    assert np.array_equal(np.stack(hx, 1), got)


@pytest.mark.parametrize("n", [1, 2, 3, 25, 26, 200])
def test_small_n_against_direct(n):
    b = ics.plummer(n, seed=11)
    s, got = _solve(b, theta=0.5)
    ref = oracle.direct(b.x, b.y, b.z, b.m)
    if n == 1:
        assert np.all(got == 0.0)
        return
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    assert _rel_dev(got, o.accel("TC")).max() <= 1e-12
    if n <= 25:
        assert _rel_dev(got, ref).max() <= 1e-13


def test_coincident_bodies_depth_cap():
    # 40 bodies at one point (depth cap 21, zero-separation pairs skipped)
    # plus a cloud around it
    rng = np.random.default_rng(0)
    p = np.concatenate([np.zeros((40, 3)) + 0.25, rng.uniform(-1, 1, (500, 3))])
    m = np.full(p.shape[0], 1.0 / p.shape[0])
    b = ics.Bodies(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m)
    s, got = _solve(b, theta=0.5)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_tree(s, o)
    _compare_lists(s, o)
    assert s.stats().depth == 21
    ref = o.accel("TC")
    assert np.all(np.isfinite(got))
    assert _rel_dev(got, ref).max() <= 1e-12


def test_all_bodies_coincident():
    n = 100
    b = ics.Bodies(np.full(n, 0.5), np.full(n, -0.25), np.full(n, 2.0), np.full(n, 0.01))
    s, got = _solve(b)
    assert np.all(got == 0.0)
    assert s.stats().depth == 21


def test_theta_to_zero_is_direct_summation():
    b = ics.plummer(600, seed=9)
    s, got = _solve(b, theta=1e-7)
    ref = oracle.direct(b.x, b.y, b.z, b.m)
    assert _rel_dev(got, ref).max() <= 1e-12


def test_invalid_inputs_rejected():
    from paper_1706_06989_gb300 import fmm
    with pytest.raises(fmm.FMMError) as e:
        _solver(theta=1.5)
    assert e.value.code == fmm.FMM_EINVAL
    b = ics.plummer(100, seed=1)
    b.x[7] = np.nan
    s = _solver(theta=0.5)
    x, y, z, m = _dev(b)
    with pytest.raises(fmm.FMMError) as e:
        s.solve(x, y, z, m)
    assert e.value.code == fmm.FMM_EINVAL
    b = ics.plummer(100, seed=1)
    b.m[3] = 0.0
    x, y, z, m = _dev(b)
    with pytest.raises(fmm.FMMError) as e:
        s.solve(x, y, z, m)
    assert e.value.code == fmm.FMM_EINVAL
    # the context stays usable
    b = ics.plummer(100, seed=1)
    x, y, z, m = _dev(b)
    s.solve(x, y, z, m)
    with pytest.raises(fmm.FMMError) as e:
        s2 = _solver(theta=0.5)
        s2.upward()
    assert e.value.code == fmm.FMM_EORDER


def test_stage_by_stage_equals_solve():
    b = ics.plummer(3000, seed=6)
    s, got = _solve(b)
    s2 = _solver(theta=0.5)
    x, y, z, m = _dev(b)
    s2.build_tree(x, y, z, m)
    s2.upward()
    s2.interact()
    s2.downward()
    a = torch.stack(s2.forces(), 1).cpu().numpy()
    assert np.array_equal(a, got)


def test_locals_l2l_consistent():
    """L2L is exact: evaluating a leaf's expansion equals evaluating the
    oracle's far field at the leaf's bodies (within rounding)."""
    b = ics.plummer(4000, seed=8)
    s, got = _solve(b)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    far = o.accel("TC", parts=oracle.PART_FAR)
    near = o.accel("TC", parts=oracle.PART_NEAR)
    assert _rel_dev(got, far + near).max() <= 1e-12


@pytest.mark.slow
def test_plummer_1m_full_size():
    """Plummer N = 1,048,576, theta = 0.5, n_crit = 25: keys, tree, geometry and
    lists bit-exact; 4096 sampled accelerations within 1e-12; balance."""
    b = ics.plummer(1 << 20, seed=0)
    s, got = _solve(b, theta=0.5)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_tree(s, o)
    _compare_lists(s, o)
    t = ics.error_subset(b.n, 4096, seed=1)
    ref = o.accel("TC", targets=t)
    assert _rel_dev(got[t], ref).max() <= 1e-12
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert fb <= 1e-13 and tb <= 1e-13


@pytest.mark.parametrize("variant", ["UC", "TC", "TCO"])
def test_mixed_precision_against_oracle(variant):
    """Mixed form: FP32 interactions on cell-relative coordinates, FP64 tree,
    moments and accumulation.  rms relative force error against the FP64
    oracle <= 1e-6; force balance <= 1e-6, and the torque balance too where
    the variant conserves it.  (UC and TC read trace-free cell records, TCO
    the raw ones.)"""
    b = ics.plummer(65536, seed=0)
    s, got = _solve(b, theta=0.5, variant=variant, precision="mixed")
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_tree(s, o)
    _compare_lists(s, o)
    t = ics.error_subset(b.n, 4096, seed=1)
    ref = o.accel(variant, targets=t)
    rel = _rel_dev(got[t], ref)
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert fb <= 1e-6, fb
    if variant != "UC":
        assert tb <= 1e-6, tb


@pytest.mark.slow
def test_mixed_precision_1m_against_oracle():
    """The mixed form at the benchmark size (Plummer N = 1,048,576, theta =
    0.5, TC): tree and lists bit-exact, rms relative deviation from the FP64
    oracle <= 1e-6 on 4,096 sampled bodies, balances <= 1e-6."""
    b = ics.plummer(1 << 20, seed=0)
    s, got = _solve(b, theta=0.5, precision="mixed")
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    _compare_tree(s, o)
    _compare_lists(s, o)
    t = ics.error_subset(b.n, 4096, seed=1)
    rel = _rel_dev(got[t], o.accel("TC", targets=t))
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert fb <= 1e-6 and tb <= 1e-6, (fb, tb)


@pytest.mark.slow
def test_mixed_precision_4m_against_oracle():
    """The mixed form at the size of the 4M-body comparison (Plummer N =
    4,194,304, theta = 0.5, TC): rms relative deviation from the FP64 oracle
    <= 1e-6 on 4,096 sampled bodies and the M2L and P2P counts the oracle's
    walk gives."""
    b = ics.plummer(1 << 22, seed=0)
    s, got = _solve(b, theta=0.5, precision="mixed")
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    st = s.stats()
    assert (st.ncell, st.n_m2l, st.n_p2p) == (o.ncell, o.n_m2l, o.n_p2p)
    t = ics.error_subset(b.n, 4096, seed=1)
    rel = _rel_dev(got[t], o.accel("TC", targets=t))
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))


@pytest.mark.slow
def test_mixed_precision_depth_capped_binary():
    """The longest FP32 sums: a binary of two dense Plummer spheres (the
    leapfrog workload's cores, N = 2,097,152) with 64 bodies thrown out to
    ~3,000 scale radii, as close encounters do.  The cube grows ~1,000-fold,
    the tree reaches the level-21 key limit and the cores' leaves hold
    hundreds of bodies, so leaf pairs and column streams are far longer than
    in a Plummer sphere.  Mixed form: rms deviation from the FP64 oracle
    <= 1e-6 on 4,096 bodies, half of them in the densest leaves."""
    b = ics.binary_plummer(1 << 21, seed=3)
    rng = np.random.default_rng(4)
    far = rng.choice(b.n, 64, replace=False)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    b.x[far], b.y[far], b.z[far] = (3000.0 * d[:, k] for k in range(3))
    s, got = _solve(b, theta=0.5, precision="mixed")
    st = s.stats()
    assert st.depth == 21
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    c = o.cells()
    leaves = np.nonzero(c.nchild == 0)[0]
    big = leaves[np.argsort(c.count[leaves])[::-1][:64]]
    assert c.count[big[0]] > 100
    dense = np.concatenate([o.cell_bodies(L) for L in big])
    rng2 = np.random.default_rng(5)
    t = np.unique(np.concatenate([rng2.choice(dense, min(2048, dense.size), replace=False),
                                  ics.error_subset(b.n, 2048, seed=6)]))
    rel = _rel_dev(got[t], o.accel("TC", targets=t))
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6, np.sqrt(np.mean(rel ** 2))


def test_mixed_precision_small_exact_cases():
    b = ics.plummer(2000, seed=0)
    s, got = _solve(b, theta=0.5, precision="mixed")
    ref = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25).accel("TC")
    rel = _rel_dev(got, ref)
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6
    s2, got2 = _solve(b, theta=0.5, precision="mixed")
    assert np.array_equal(got, got2)


def test_direct_diagnostic_matches_oracle():
    b = ics.plummer(20000, seed=21)
    s = _solver(theta=0.5)
    x, y, z, m = _dev(b)
    t = ics.error_subset(b.n, 300, seed=2)
    a = torch.stack(s.direct(x, y, z, m, t), 1).cpu().numpy()
    ref = oracle.direct(b.x, b.y, b.z, b.m, targets=t)
    assert _rel_dev(a, ref).max() <= 1e-14
    a2 = torch.stack(s.direct(x, y, z, m, t), 1).cpu().numpy()
    assert np.array_equal(a, a2)


def test_balance_diagnostic_matches_oracle():
    b = ics.plummer(50000, seed=22)
    s, got = _solve(b, variant="UC")
    x, y, z, m = _dev(b)
    g = torch.from_numpy(got).cuda()
    fb, tb = s.balance(x, y, z, m, g[:, 0].contiguous(), g[:, 1].contiguous(), g[:, 2].contiguous())
    ofb, otb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert abs(tb - otb) <= 1e-3 * otb  # UC: a clear torque imbalance, same value
    assert fb <= 1e-13 and ofb <= 1e-13


def test_lists_when_the_walk_outgrows_its_buffers():
    """A small opening angle on a uniform cube makes the frontier and the
    near-field list outgrow their first buffers (at most 32 n and 48 n
    pairs): every leaf pair is summed directly.  The generation is flagged,
    the buffers grow and the generation runs again.  Lists must still match
    the oracle bit for bit, and a second solve (buffers already large) must
    give the same accelerations."""
    b = ics.uniform_cube(20000, seed=11)
    s, a = _solve(b, theta=0.05)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.05, 25)
    st = s.stats()
    assert st.n_p2p > 48 * b.n  # beyond the first P2P buffer
    m2l, p2p, slf = s.export_lists()
    om2l, op2p, oslf = o.lists()
    assert np.array_equal(_canon_pairs(m2l.cpu().numpy()), _canon_pairs(om2l))
    assert np.array_equal(_canon_pairs(p2p.cpu().numpy()), _canon_pairs(op2p))
    assert np.array_equal(np.sort(slf.cpu().numpy()), np.sort(oslf))
    ref = o.accel("TC")
    assert _rel_dev(a, ref).max() <= 1e-12
    x, y, z, m = _dev(b)
    a2 = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    assert np.array_equal(a, a2)


_CHUNK_REF = {}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_long_column_streams_are_split(precision):
    """At a small opening angle every leaf sums directly with most others, so
    its column stream runs to tens of thousands of bodies and is cut into
    chunks (at most 2,048 columns in FP64, 4,096 in FP32) handled by separate
    warps (the later chunks' A-side partials are added in chunk order
    afterwards).  The accelerations must still match the oracle."""
    b = ics.uniform_cube(40000, seed=12)
    s, a = _solve(b, theta=0.05, precision=precision)
    st = s.stats()
    # mean column stream of a leaf (body pairs / leaves / mean leaf size) beyond one chunk
    assert st.p2p_body_pairs / st.nleaf / (b.n / st.nleaf) > 16384
    if "ref" not in _CHUNK_REF:
        _CHUNK_REF["ref"] = oracle.Oracle(b.x, b.y, b.z, b.m, 0.05, 25).accel("TC")
    ref = _CHUNK_REF["ref"]
    dev = _rel_dev(a, ref)
    if precision == "fp64":
        assert dev.max() <= 1e-12
    else:
        assert np.sqrt(np.mean(dev ** 2)) <= 1e-6
    x, y, z, m = _dev(b)
    a2 = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    assert np.array_equal(a, a2)


@pytest.mark.parametrize("theta,n_crit", [(1.0, 25), (0.5, 1), (0.5, 64), (0.7, 5000)])
def test_opening_angle_and_leaf_size_extremes(theta, n_crit):
    """theta at its largest (Sec. 2 allows 0 < theta <= 1), one body per leaf,
    large leaves, and a tree that is a single leaf: tree, lists and FP64
    accelerations against the oracle."""
    b = ics.plummer(3000, seed=13)
    s, a = _solve(b, theta=theta, n_crit=n_crit)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, theta, n_crit)
    _compare_tree(s, o)
    m2l, p2p, slf = s.export_lists()
    om2l, op2p, oslf = o.lists()
    assert np.array_equal(_canon_pairs(m2l.cpu().numpy()), _canon_pairs(om2l))
    assert np.array_equal(_canon_pairs(p2p.cpu().numpy()), _canon_pairs(op2p))
    assert np.array_equal(np.sort(slf.cpu().numpy()), np.sort(oslf))
    assert _rel_dev(a, o.accel("TC")).max() <= 1e-12
    if n_crit >= b.n:
        assert s.stats().ncell == 1


def test_bounded_wait_returns_timeout_and_context_survives():
    """The walk's look-back waits for earlier blocks with a poll limit.  The
    test hook makes a block wait for a block that does not exist: the call
    must return FMM_ETIMEOUT (not hang), and a solve on the same context must
    still match the oracle."""
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(2000, seed=14)
    s = _solver(theta=0.5)
    assert s.debug_walk_wait_timeout() == fmm.FMM_ETIMEOUT
    x, y, z, m = _dev(b)
    a = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    ref = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25).accel("TC")
    assert _rel_dev(a, ref).max() <= 1e-12


def test_tree_levels_on_a_reused_context():
    """The tree is built in batches of levels sized by the previous tree's
    depth.  One context solves a deep system, a shallow one, the deep one
    again and then a system whose tree outgrows the cell room of the first
    build (one body per leaf): every tree, list set and FP64 result must
    match the oracle."""
    from paper_1706_06989_gb300 import fmm
    deep = ics.plummer(6000, seed=21)
    shallow = ics.uniform_cube(1500, seed=22)
    s = fmm.FMM(theta=0.5, n_crit=25, variant="TC", precision="fp64")
    depths = []
    for b, n_crit in ((deep, 25), (shallow, 25), (deep, 25), (deep, 1)):
        s.set_opts(n_crit=n_crit)
        x, y, z, m = _dev(b)
        a = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
        o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, n_crit)
        _compare_tree(s, o)
        m2l, p2p, slf = s.export_lists()
        om2l, op2p, oslf = o.lists()
        assert np.array_equal(_canon_pairs(m2l.cpu().numpy()), _canon_pairs(om2l))
        assert np.array_equal(_canon_pairs(p2p.cpu().numpy()), _canon_pairs(op2p))
        assert _rel_dev(a, o.accel("TC")).max() <= 1e-12
        depths.append(s.stats().depth)
    assert depths[0] > depths[1] and depths[3] > depths[0]
    assert s.stats().ncell > 6000 // 2 + 64  # beyond the first build's cell room
