"""a13: a solve as one CUDA-graph launch (fmm_set_graph), through the C ABI.

The graph is captured from the host code of a plain solve; replays must give
the plain solve's results bit for bit (coordinates and masses are read from
the device at every replay), fall back to a plain solve when a size the
launches were captured with changes, and capture again once a plan repeats.
"""
import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _solver(**kw):
    from paper_1706_06989_gb300 import fmm
    return fmm.FMM(**kw)


def _out(n):
    return tuple(torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))


def _acc(out):
    return torch.stack(out, 1).cpu().numpy()


def _stats_tuple(st):
    return (st.ncell, st.nleaf, st.depth, st.n_m2l, st.n_p2p, st.n_self, st.p2p_body_pairs)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forest_replay_is_bit_identical(precision):
    off, b = ics.ensemble(nsys=48, seed=5, nmin=64, nmax=6000)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    plain = _solver(theta=0.5, precision=precision)
    ref = _acc(plain.solve_batch(x, y, z, m, off))
    ref_st = _stats_tuple(plain.stats())

    g = _solver(theta=0.5, precision=precision)
    g.set_graph(True)
    out = _out(b.n)
    # first solve: plain, then captured
    assert np.array_equal(_acc(g.solve_batch(x, y, z, m, off, out=out)), ref)
    gs = g.graph_stats()
    assert gs["captures"] == 1 and gs["replays"] == 0 and gs["kernels"] > 50, gs
    for k in range(3):
        for o in out:
            o.fill_(float("nan"))
        assert np.array_equal(_acc(g.solve_batch(x, y, z, m, off, out=out)), ref), k
        assert _stats_tuple(g.stats()) == ref_st
    gs = g.graph_stats()
    assert gs["replays"] == 3 and gs["fallbacks"] == 0 and gs["captures"] == 1
    assert g.stats().launches == gs["kernels"]

    # new masses, same sizes: the replay solves the new system (a uniform
    # factor keeps centres, R_max and so every list)
    m2 = m * 2.0
    m.copy_(m2)
    ref2 = _acc(plain.solve_batch(x, y, z, m, off))
    assert np.array_equal(_acc(g.solve_batch(x, y, z, m, off, out=out)), ref2)
    assert g.graph_stats()["replays"] == 4


def test_replay_falls_back_when_sizes_change_and_recaptures():
    off, b = ics.ensemble(nsys=16, seed=6, nmin=256, nmax=5000)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    plain = _solver(theta=0.5)
    g = _solver(theta=0.5)
    g.set_graph(True)
    out = _out(b.n)
    g.solve_batch(x, y, z, m, off, out=out)
    assert g.graph_stats()["captures"] == 1
    # other coordinates (fresh draws of the same sizes): another tree and
    # other lists
    parts = [ics.plummer(int(off[k + 1] - off[k]), seed=5000 + k) for k in range(len(off) - 1)]
    for v, f in zip((x, y, z), ("x", "y", "z")):
        v.copy_(torch.from_numpy(np.concatenate([getattr(p, f) for p in parts])).cuda())
    ref = _acc(plain.solve_batch(x, y, z, m, off))
    assert np.array_equal(_acc(g.solve_batch(x, y, z, m, off, out=out)), ref)
    gs = g.graph_stats()
    assert gs["fallbacks"] == 1 and gs["captures"] == 1 and gs["replays"] == 0
    assert _stats_tuple(g.stats()) == _stats_tuple(plain.stats())
    # the same system again: its plan repeats, so it is captured ...
    assert np.array_equal(_acc(g.solve_batch(x, y, z, m, off, out=out)), ref)
    assert g.graph_stats()["captures"] == 2
    # ... and replayed
    assert np.array_equal(_acc(g.solve_batch(x, y, z, m, off, out=out)), ref)
    gs = g.graph_stats()
    assert gs["replays"] == 1 and gs["fallbacks"] == 1


def test_single_system_replay_matches_oracle():
    b = ics.plummer(30000, seed=21)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    g = _solver(theta=0.5, variant="TCO")
    g.set_graph(True)
    out = _out(b.n)
    first = _acc(g.solve(x, y, z, m, out=out))
    second = _acc(g.solve(x, y, z, m, out=out))
    assert g.graph_stats()["replays"] == 1
    assert np.array_equal(first, second)
    t = ics.error_subset(b.n, 2000, seed=4)
    ref = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25).accel("TCO", targets=t)
    rel = np.linalg.norm(second[t] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() <= 1e-12


def test_options_change_recaptures():
    b = ics.plummer(20000, seed=22)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    g = _solver(theta=0.5)
    g.set_graph(True)
    out = _out(b.n)
    g.solve(x, y, z, m, out=out)
    g.set_opts(theta=0.7)
    a7 = _acc(g.solve(x, y, z, m, out=out))
    assert g.graph_stats()["captures"] == 2
    p = _solver(theta=0.7)
    assert np.array_equal(a7, _acc(p.solve(x, y, z, m)))
    assert np.array_equal(_acc(g.solve(x, y, z, m, out=out)), a7)
    assert g.graph_stats()["replays"] == 1


def test_invalid_input_after_capture_is_reported():
    """A NaN coordinate after the capture: the replay's first check fails,
    the call solves plainly and returns the plain solve's error."""
    from paper_1706_06989_gb300 import fmm
    b = ics.plummer(5000, seed=23)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    g = _solver(theta=0.5)
    g.set_graph(True)
    out = _out(b.n)
    g.solve(x, y, z, m, out=out)
    x[17] = float("nan")
    with pytest.raises(fmm.FMMError) as e:
        g.solve(x, y, z, m, out=out)
    assert e.value.code == fmm.FMM_EINVAL
    assert g.graph_stats()["fallbacks"] == 1
    x[17] = float(b.x[17])
    ref = _acc(_solver(theta=0.5).solve(x, y, z, m))
    assert np.array_equal(_acc(g.solve(x, y, z, m, out=out)), ref)


def test_leapfrog_with_graph_equals_plain():
    """An integration changes the positions every step: a replay solves
    the step when its sizes match the capture, otherwise the step is solved
    plainly; either way bit-identical to the plain path."""
    b = ics.plummer(8000, seed=24, velocities=True)
    res = []
    for graph in (False, True):
        s = _solver(theta=0.5)
        s.set_graph(graph)
        st = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.vx, b.vy, b.vz)]
        m = torch.from_numpy(b.m).cuda()
        s.leapfrog(*st, m, dt=1e-2, nsteps=4, record=False)
        res.append(torch.stack(st, 1).cpu().numpy())
        if graph:
            gs = s.graph_stats()
            assert gs["captures"] >= 1 and gs["replays"] + gs["fallbacks"] + gs["captures"] >= 2
    assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_softened_replay_is_bit_identical(precision):
    """Softening selects the kernels on raw moments; the captured graph
    holds them and replays bit-identically."""
    b = ics.plummer(20000, seed=25)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    p = _solver(theta=0.5, precision=precision)
    p.set_softening(0.01)
    ref = _acc(p.solve(x, y, z, m))
    g = _solver(theta=0.5, precision=precision)
    g.set_softening(0.01)
    g.set_graph(True)
    out = _out(b.n)
    assert np.array_equal(_acc(g.solve(x, y, z, m, out=out)), ref)
    assert np.array_equal(_acc(g.solve(x, y, z, m, out=out)), ref)
    gs = g.graph_stats()
    assert gs["replays"] == 1 and gs["captures"] == 1


@pytest.mark.parametrize("case", ["one", "two", "coincident", "forest_with_singletons"])
def test_degenerate_systems_replay(case):
    """Solves without accepted pairs or without leaf pairs skip stages and
    read back less; their graphs replay bit-identically too."""
    rng = np.random.default_rng(11)
    off = None
    if case == "one":
        p, m = np.zeros((1, 3)), np.ones(1)
    elif case == "two":
        p, m = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.25]]), np.array([1.0, 2.0])
    elif case == "coincident":
        p, m = np.tile([0.3, -0.2, 0.1], (40, 1)), rng.uniform(0.5, 1.5, 40)
    else:
        sizes = [1, 500, 1, 1, 2, 3000, 1]
        p = np.concatenate([rng.normal(size=(k, 3)) for k in sizes])
        m = rng.uniform(0.5, 1.5, p.shape[0])
        off = np.concatenate([[0], np.cumsum(sizes)])
    b = ics.Bodies(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m)
    x, y, z, mm = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.m))
    plain = _solver(theta=0.5)
    g = _solver(theta=0.5)
    g.set_graph(True)
    out = _out(b.n)
    if off is None:
        ref = _acc(plain.solve(x, y, z, mm))
        runs = [_acc(g.solve(x, y, z, mm, out=out)) for _ in range(3)]
    else:
        ref = _acc(plain.solve_batch(x, y, z, mm, off))
        runs = [_acc(g.solve_batch(x, y, z, mm, off, out=out)) for _ in range(3)]
    for r in runs:
        assert np.array_equal(r, ref)
    gs = g.graph_stats()
    assert gs["captures"] == 1 and gs["replays"] == 2, gs
