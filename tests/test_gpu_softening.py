"""Softened Green's function on the GPU (Sec. 4: the correction holds for any
G of the distance alone), against the oracle's softened evaluation: FP64
accelerations within 1e-12 per body, the mixed form within 1e-6 rms, the
softened direct sums, and the torque of a single accepted pair cancelled with
softening as without."""
import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(b):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))


def _rel(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("variant", ["UC", "TC", "TCO"])
def test_softened_fp64_matches_oracle(variant):
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(6000, seed=41)
    eps = 0.02
    s = fmm.FMM(theta=0.5, variant=variant)
    s.set_softening(eps)
    a = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25, softening=eps)
    assert s.stats().n_m2l == o.n_m2l  # the lists do not depend on eps
    ref = o.accel(variant)
    assert _rel(a, ref).max() <= 1e-12
    # softening changes the answer (the test is not passing on unsoftened code)
    unsoft = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25).accel(variant)
    assert np.sqrt(np.mean(_rel(unsoft, ref) ** 2)) > 1e-4
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, a)
    assert fb <= 1e-13
    if variant != "UC":
        assert tb <= 1e-13


def test_softened_mixed_matches_oracle():
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(65536, seed=42)
    eps = 0.01
    s = fmm.FMM(theta=0.5, variant="TC", precision="mixed")
    s.set_softening(eps)
    a = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25, softening=eps)
    t = ics.error_subset(b.n, 4096, seed=1)
    rel = _rel(a[t], o.accel("TC", targets=t))
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, a)
    assert fb <= 1e-6 and tb <= 1e-6


def test_softened_direct_diagnostic():
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(5000, seed=43)
    s = fmm.FMM()
    s.set_softening(0.05)
    tg = ics.error_subset(b.n, 300, seed=2)
    x, y, z, m = _dev(b)
    g = torch.stack(s.direct(x, y, z, m, tg), 1).cpu().numpy()
    ref = oracle.direct(b.x, b.y, b.z, b.m, targets=tg, eps=0.05)
    assert np.abs(g - ref).max() <= 1e-14 * np.abs(ref).max()


def test_single_softened_pair_torque_cancelled():
    """Two clusters of 20 bodies that the walk accepts as one M2L pair (each
    cluster is one leaf), softening comparable with their size: the net
    torque of the solve is that pair's torque (the clusters' own direct sums
    conserve it exactly).  TC and TCO cancel it, UC leaves it."""
    from paper_1706_06989_gb300 import fmm
    rng = np.random.default_rng(7)
    p = np.concatenate([rng.normal(size=(20, 3)) * [0.3, 0.1, 0.2] + [-2.0, -2.0, -2.0],
                        rng.normal(size=(20, 3)) * [0.1, 0.25, 0.15] + [2.0, 2.0, 2.0]])
    m = rng.uniform(0.5, 1.5, 40)
    b = ics.Bodies(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m)
    torques = {}
    for v in ("UC", "TC", "TCO"):
        s = fmm.FMM(theta=1.0, variant=v)
        s.set_softening(0.5)
        a = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
        st = s.stats()
        assert st.n_m2l == 1 and st.n_p2p == 0
        ref = oracle.Oracle(b.x, b.y, b.z, b.m, 1.0, 25, softening=0.5).accel(v)
        assert _rel(a, ref).max() <= 1e-12
        torques[v] = oracle.balance(b.x, b.y, b.z, b.m, a)[1]
    assert torques["UC"] > 1e-8
    assert torques["TC"] <= 1e-14 and torques["TCO"] <= 1e-14


def test_softening_arguments():
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(3000, seed=44)
    s = fmm.FMM(theta=0.5)
    with pytest.raises(fmm.FMMError):
        s.set_softening(-1.0)
    with pytest.raises(fmm.FMMError):
        s.set_softening(float("inf"))
    a0 = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    s.set_softening(0.1)
    s.solve(*_dev(b))
    s.set_softening(0.0)  # back to the unsoftened method, bit for bit
    a1 = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    assert np.array_equal(a0, a1)
    s4 = fmm.FMM(theta=0.5, order_P=4)
    s4.set_softening(0.1)
    with pytest.raises(fmm.FMMError) as e:
        s4.solve(*_dev(b))
    assert e.value.code == fmm.FMM_EUNSUPPORTED


@pytest.mark.parametrize("variant", ["UC", "TCO"])
def test_softened_mixed_other_variants(variant):
    """The mixed form's raw-moment records (softened) for the other two
    variants: rms <= 1e-6 against the softened oracle, forces balanced, and
    the torque too where the variant conserves it."""
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(40000, seed=45)
    eps = 0.01
    s = fmm.FMM(theta=0.5, variant=variant, precision="mixed")
    s.set_softening(eps)
    a = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25, softening=eps)
    t = ics.error_subset(b.n, 3000, seed=2)
    rel = _rel(a[t], o.accel(variant, targets=t))
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, a)
    assert fb <= 1e-6
    if variant != "UC":
        assert tb <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_softened_forest_equals_one_solve_per_system(precision):
    """Forests honour the softening: each system of the forest is
    bit-identical to its own softened solve, and matches the oracle."""
    from paper_1706_06989_gb300 import fmm
    off, b = ics.ensemble(nsys=6, seed=9, nmin=300, nmax=3000)
    eps = 0.02
    s = fmm.FMM(theta=0.5, precision=precision)
    s.set_softening(eps)
    x, y, z, m = _dev(b)
    got = torch.stack(s.solve_batch(x, y, z, m, off), 1).cpu().numpy()
    for k in range(len(off) - 1):
        sl = slice(int(off[k]), int(off[k + 1]))
        one = torch.stack(s.solve(x[sl].contiguous(), y[sl].contiguous(), z[sl].contiguous(),
                                  m[sl].contiguous()), 1).cpu().numpy()
        assert np.array_equal(one, got[sl]), k
    if precision == "fp64":
        sl = slice(int(off[0]), int(off[1]))
        ref = oracle.Oracle(b.x[sl], b.y[sl], b.z[sl], b.m[sl], 0.5, 25, softening=eps).accel("TC")
        assert _rel(got[sl], ref).max() <= 1e-12
