"""a7' and the higher orders: the general-order expansion of App. A on the
GPU (P = 4, 5 generated; P = 6, 7, 8 table-driven; FP64) against the
oracle's general-order path, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solve(b, P, variant, theta=0.6, n_crit=16):
    from paper_1706_06989_gb300 import fmm
    s = fmm.FMM(theta=theta, n_crit=n_crit, variant=variant, order_P=P)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    a = torch.stack(s.solve(x, y, z, m), 1).cpu().numpy()
    return s, a


def _rel(a, r):
    return np.linalg.norm(a - r, axis=1) / np.linalg.norm(r, axis=1)


@pytest.mark.parametrize("P", [4, 5])
@pytest.mark.parametrize("variant", ["UC", "TC", "TCO"])
def test_general_order_matches_oracle(P, variant):
    b = ics.plummer(3000, seed=17)
    s, got = _solve(b, P, variant)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.6, 16, P=P)
    assert s.stats().n_m2l == o.n_m2l and s.stats().ncell == o.ncell
    ref = o.accel(variant, generic=True)
    assert _rel(got, ref).max() <= 1e-12
    mom = s.export_moments().cpu().numpy()
    _, _, R, omom = o.geometry()
    assert mom.shape == omom.shape
    M = omom[:, 0]
    for n_ord in range(1, P + 1):
        lo, hi = n_ord * (n_ord + 1) * (n_ord + 2) // 6, (n_ord + 1) * (n_ord + 2) * (n_ord + 3) // 6
        tol = 1e-12 * (M * np.maximum(R, 1e-300) ** n_ord)[:, None] + 1e-300
        assert np.all(np.abs(mom[:, lo:hi] - omom[:, lo:hi]) <= tol + 1e-13 * np.abs(omom[:, lo:hi])), n_ord
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert fb <= 1e-13
    if variant != "UC":
        assert tb <= 1e-13


# the oracle's general order sums over full index tuples (3^n terms per
# order), so the cases shrink as P grows
_HIGH = {6: (400, 0.6, 8, ("UC", "TC", "TCO")), 7: (400, 0.6, 8, ("TC", "TCO")), 8: (250, 0.8, 8, ("TC",))}


@pytest.mark.parametrize("P,variant", [(P, v) for P, (_, _, _, vs) in _HIGH.items() for v in vs])
def test_table_driven_orders_match_oracle(P, variant):
    n, theta, n_crit, _ = _HIGH[P]
    b = ics.plummer(n, seed=17)
    s, got = _solve(b, P, variant, theta=theta, n_crit=n_crit)
    o = oracle.Oracle(b.x, b.y, b.z, b.m, theta, n_crit, P=P)
    assert s.stats().n_m2l == o.n_m2l and s.stats().ncell == o.ncell
    ref = o.accel(variant, generic=True)
    assert _rel(got, ref).max() <= 1e-12, _rel(got, ref).max()
    mom = s.export_moments().cpu().numpy()
    _, _, R, omom = o.geometry()
    assert mom.shape == omom.shape
    M = omom[:, 0]
    for n_ord in range(1, P + 1):
        lo, hi = n_ord * (n_ord + 1) * (n_ord + 2) // 6, (n_ord + 1) * (n_ord + 2) * (n_ord + 3) // 6
        tol = 1e-12 * (M * np.maximum(R, 1e-300) ** n_ord)[:, None] + 1e-300
        assert np.all(np.abs(mom[:, lo:hi] - omom[:, lo:hi]) <= tol + 1e-13 * np.abs(omom[:, lo:hi])), n_ord
    fb, tb = oracle.balance(b.x, b.y, b.z, b.m, got)
    assert fb <= 1e-13
    if variant != "UC":
        assert tb <= 1e-13


def test_error_falls_with_order_through_eight():
    b = ics.plummer(3000, seed=19)
    ref = oracle.direct(b.x, b.y, b.z, b.m)
    err = {}
    for P in (3, 4, 5, 6, 7, 8):
        _, a = _solve(b, P, "TC", theta=0.6, n_crit=16)
        err[P] = np.sqrt(np.mean(_rel(a, ref) ** 2))
    assert all(err[P + 1] < err[P] for P in range(3, 8)), err


def test_higher_order_reduces_error_on_gpu():
    b = ics.plummer(4000, seed=19)
    ref = oracle.direct(b.x, b.y, b.z, b.m)
    err = {}
    for P in (3, 4, 5):
        _, a = _solve(b, P, "TC", theta=0.6, n_crit=16)
        err[P] = np.sqrt(np.mean(_rel(a, ref) ** 2))
    assert err[5] < err[4] < err[3]


def test_orders_above_three_need_fp64():
    from paper_1706_06989_gb300 import fmm
    with pytest.raises(fmm.FMMError) as e:
        fmm.FMM(order_P=4, precision="mixed")
    assert e.value.code == fmm.FMM_EUNSUPPORTED
    with pytest.raises(fmm.FMMError):
        fmm.FMM(order_P=9)
