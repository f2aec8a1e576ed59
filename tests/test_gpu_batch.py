"""a13: ensembles of independent systems solved as one forest in one launch
sequence (through the C ABI), the near field's leaf tile, and the autotuner
over leaf size and tile."""
import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(**kw):
    from paper_1706_06989_gb300 import fmm
    return fmm.FMM(**kw)


def _dev(b):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))


def _ensemble(nsys, seed, nmin=1, nmax=3000):
    return ics.ensemble(nsys=nsys, seed=seed, nmin=nmin, nmax=nmax)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forest_equals_one_solve_per_system(precision):
    off, b = _ensemble(24, seed=3, nmin=1, nmax=4000)
    s = _solver(theta=0.5, precision=precision)
    x, y, z, m = _dev(b)
    got = torch.stack(s.solve_batch(x, y, z, m, off), 1).cpu().numpy()
    st = s.stats()
    ncell = n_m2l = n_p2p = 0
    for k in range(len(off) - 1):
        sl = slice(int(off[k]), int(off[k + 1]))
        one = torch.stack(s.solve(x[sl].contiguous(), y[sl].contiguous(), z[sl].contiguous(),
                                  m[sl].contiguous()), 1).cpu().numpy()
        assert np.array_equal(one, got[sl]), k
        so = s.stats()
        ncell += so.ncell
        n_m2l += so.n_m2l
        n_p2p += so.n_p2p
    assert (st.ncell, st.n_m2l, st.n_p2p) == (ncell, n_m2l, n_p2p)


def test_forest_matches_oracle_per_system():
    off, b = _ensemble(12, seed=8, nmin=1, nmax=2500)
    s = _solver(theta=0.6, variant="TCO")
    x, y, z, m = _dev(b)
    got = torch.stack(s.solve_batch(x, y, z, m, off), 1).cpu().numpy()
    for k in range(len(off) - 1):
        sl = slice(int(off[k]), int(off[k + 1]))
        if off[k + 1] - off[k] == 1:
            assert np.all(got[sl] == 0.0)
            continue
        ref = oracle.Oracle(b.x[sl], b.y[sl], b.z[sl], b.m[sl], 0.6, 25).accel("TCO")
        rel = np.linalg.norm(got[sl] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert rel.max() <= 1e-12, (k, rel.max())


def test_forest_rejects_bad_offsets():
    from paper_1706_06989_gb300 import fmm
    off, b = _ensemble(4, seed=1, nmin=10, nmax=50)
    s = _solver()
    x, y, z, m = _dev(b)
    bad = off.copy()
    bad[2] = bad[1]  # an empty system
    with pytest.raises(fmm.FMMError) as e:
        s.solve_batch(x, y, z, m, bad)
    assert e.value.code == fmm.FMM_EINVAL
    s.solve_batch(x, y, z, m, off)  # still usable


def test_autotune_picks_a_candidate_and_restores_options():
    off, b = _ensemble(16, seed=5, nmin=500, nmax=5000)
    s = _solver(theta=0.5, n_crit=25)
    x, y, z, m = _dev(b)
    best, ms = s.autotune_ncrit(x, y, z, m, off, candidates=(16, 25, 32, 64), reps=2)
    assert best in (16, 25, 32, 64) and all(v > 0 for v in ms.values())
    assert ms[best] == min(ms.values())
    assert s.opts.n_crit == 25


@pytest.mark.parametrize("tile", [8, 32])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_leaf_tiles_match_oracle(tile, precision):
    """The near field's leaf tile (rows staged per pass) changes only the
    order of the work: with leaves of up to 64 bodies (several passes at
    tile 8 and 16, one at 32) the FP64 form stays within 1e-12 of the oracle
    and the mixed form within 1e-6 rms."""
    b = ics.plummer(20000, seed=23)
    s = _solver(theta=0.5, n_crit=64, precision=precision)
    s.set_tile(tile)
    got = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    ref = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 64).accel("TC")
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    if precision == "fp64":
        assert rel.max() <= 1e-12
    else:
        assert np.sqrt(np.mean(rel ** 2)) <= 1e-6


def test_leaf_tile_rejects_other_sizes():
    from paper_1706_06989_gb300 import fmm
    s = _solver()
    for bad in (0, 4, 24, 64):
        with pytest.raises(fmm.FMMError) as e:
            s.set_tile(bad)
        assert e.value.code == fmm.FMM_EINVAL


def test_autotune_over_leaf_size_and_tile():
    off, b = _ensemble(16, seed=6, nmin=500, nmax=5000)
    s = _solver(theta=0.5, n_crit=25)
    x, y, z, m = _dev(b)
    bn, bt, table = s.autotune(x, y, z, m, off, ncrit=(16, 32), tiles=(8, 16, 32), reps=2)
    assert set(table) == {(a, t) for a in (16, 32) for t in (8, 16, 32)}
    assert all(v > 0 for v in table.values())
    assert table[(bn, bt)] == min(table.values())
    assert s.opts.n_crit == 25
    # the chosen setting solves the ensemble like the default one (FP64)
    ref = torch.stack(s.solve_batch(x, y, z, m, off), 1).cpu().numpy()
    s.set_opts(n_crit=bn)
    s.set_tile(bt)
    got = torch.stack(s.solve_batch(x, y, z, m, off), 1).cpu().numpy()
    s.set_opts(n_crit=25)
    s.set_tile(16)
    again = torch.stack(s.solve_batch(x, y, z, m, off), 1).cpu().numpy()
    assert np.array_equal(ref, again)
    rel = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.sqrt(np.mean(rel ** 2)) < 1e-2  # another n_crit: the same method, another tree
