"""The paper's own test problem (Sec. 3) on the GPU: a double white dwarf of
two Lane-Emden polytropes (accretor index 3, mass 1; donor index 1.5, mass
0.2, filling its Roche lobe), sampled by equal-mass bodies.  Against the
oracle, and the Sec. 3 findings on it: force balance at rounding for every
variant, torque balance at rounding for TC and TCO only, TC as accurate as
UC, TCO less accurate."""
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
def test_dwd_fp64_matches_oracle(variant):
    from paper_1706_06989_gb300 import fmm
    b = ics.dwd(30000, seed=2)
    s = fmm.FMM(theta=0.5, variant=variant)
    a = torch.stack(s.solve(*_dev(b)), 1).cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    st = s.stats()
    assert (st.ncell, st.n_m2l, st.n_p2p) == (o.ncell, o.n_m2l, o.n_p2p)
    assert _rel(a, o.accel(variant)).max() <= 1e-12


def test_dwd_sec3_findings_and_mixed_form():
    from paper_1706_06989_gb300 import fmm
    b = ics.dwd(262144, seed=3)
    x, y, z, m = _dev(b)
    t = ics.error_subset(b.n, 2048, seed=1)
    s = fmm.FMM(theta=0.5)
    ref = torch.stack(s.direct(x, y, z, m, t), 1).cpu().numpy()
    res = {}
    for v in ("UC", "TC", "TCO"):
        s.set_opts(variant=v)
        out = s.solve(x, y, z, m)
        a = torch.stack(out, 1).cpu().numpy()
        res[v] = (s.balance(x, y, z, m, *out), np.mean(_rel(a[t], ref)))
    for v in res:
        assert res[v][0][0] <= 1e-15
    assert res["TC"][0][1] <= 1e-15 and res["TCO"][0][1] <= 1e-15
    assert res["UC"][0][1] > 1e3 * res["TC"][0][1]
    assert abs(res["TC"][1] - res["UC"][1]) < 0.2 * res["UC"][1]
    assert res["TCO"][1] > res["TC"][1]
    # the mixed form against the FP64 oracle on the same bodies
    sm = fmm.FMM(theta=0.5, precision="mixed")
    a = torch.stack(sm.solve(x, y, z, m), 1).cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, 0.5, 25)
    rel = _rel(a[t], o.accel("TC", targets=t))
    assert np.sqrt(np.mean(rel ** 2)) <= 1e-6
