"""fmm_balance_noalloc: the Sec. 3 balance check for callers that cannot
allocate device memory (their device memory comes from their own fixed pool,
or their time-step loop must not stall on cudaMalloc / cudaFree).  It keeps its
scratch in a fixed array inside the library and takes no context.

Checked here through the C ABI against the allocating entry point
(fmm_balance), on two calls in a row.  This file is collected last on
purpose: it must pass alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FMM_ESIZE = -7
MAX_BODIES = 4_194_304


def _entry():
    from paper_1706_06989_gb300 import fmm
    f = fmm.load().fmm_balance_noalloc
    P = ctypes.c_void_p
    f.argtypes = [P] * 7 + [ctypes.c_int64, P, P]
    f.restype = ctypes.c_int
    return f


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _cases():
    from paper_1706_06989_gb300 import fmm, ics
    dev = torch.device("cuda")
    b = ics.plummer(300_000, seed=31)
    x, y, z, m = (torch.from_numpy(a).to(dev) for a in (b.x, b.y, b.z, b.m))
    solver = fmm.FMM(theta=0.5, variant="UC")
    acc = solver.solve(x, y, z, m)
    rng = np.random.default_rng(5)
    rand = tuple(torch.from_numpy(rng.normal(size=b.n)).to(dev) for _ in range(3))
    return solver, (x, y, z, m), [("uc_solve", acc), ("random", rand)]


def test_noalloc_balance_matches_allocating_entry_point():
    f = _entry()
    solver, (x, y, z, m), cases = _cases()
    stream = torch.cuda.current_stream()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for name, (ax, ay, az) in cases:
        ref = solver.balance(x, y, z, m, ax, ay, az)
        for call in range(2):
            out.fill_(-1.0)
            rc = f(_p(x), _p(y), _p(z), _p(m), _p(ax), _p(ay), _p(az), x.shape[0], _p(out),
                   ctypes.c_void_p(stream.cuda_stream))
            assert rc == 0, (name, call, rc)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for k in range(2):
                # both are compensated FP64 sums, grouped differently
                assert abs(got[k] - ref[k]) <= 1e-12 * ref[k] + 1e-16, (name, call, k, got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = _entry()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    rc = f(*([_p(t)] * 7), MAX_BODIES + 1, _p(out), None)
    assert rc == FMM_ESIZE
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == -1.0)  # nothing was launched
