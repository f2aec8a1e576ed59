"""The Sec. 3 experiment grid on the GPU against the oracle: the solves that
bench.py's theta sweep times (UC, TC and TCO at the ends of its theta range)
and the diagnostics it reports (mean relative force and torque errors against
exact direct sums, the net force and torque balance)."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

_REF = {}


def _case():
    if "b" not in _REF:
        b = ics.plummer(12000, seed=31)
        tg = ics.error_subset(b.n, 1024, seed=1)
        _REF["b"], _REF["tg"] = b, tg
        _REF["direct"] = oracle.direct(b.x, b.y, b.z, b.m, targets=tg)
    return _REF["b"], _REF["tg"], _REF["direct"]


@pytest.mark.parametrize("theta", [0.2, 1.0])
@pytest.mark.parametrize("variant", ["UC", "TC", "TCO"])
def test_sweep_point_matches_oracle(theta, variant):
    from paper_1706_06989_gb300 import fmm
    b, tg, exact = _case()
    dev = torch.device("cuda", 0)
    x, y, z, m = (torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (b.x, b.y, b.z, b.m))
    s = fmm.FMM(theta=0.5, n_crit=25, variant="TC", precision="fp64")
    s.set_opts(theta=theta, variant=variant)  # the sweep reuses one context
    out = s.solve(x, y, z, m)
    a = torch.stack(out, 1).cpu().numpy()
    o = oracle.Oracle(b.x, b.y, b.z, b.m, theta, 25)
    ref = o.accel(variant)
    dev_ = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert dev_.max() <= 1e-12, dev_.max()
    # the diagnostics the sweep reports: GPU direct sums and the torque error
    # metric on GPU forces against the oracle's on its own forces
    tgd = torch.as_tensor(tg, device=dev)
    gd = torch.stack(s.direct(x, y, z, m, tgd), 1).cpu().numpy()
    assert np.abs(gd - exact).max() <= 1e-14 * np.abs(exact).max()
    pos = b.pos()[tg]
    te_gpu = bench.torque_errors(pos, a[tg], gd).numpy()
    te_orc = oracle.torque_errors(pos, ref[tg], exact)
    assert abs(te_gpu.mean() - te_orc["mean"]) <= 1e-9 * te_orc["mean"]
    fe_gpu = np.linalg.norm(a[tg] - gd, axis=1) / np.linalg.norm(gd, axis=1)
    assert abs(fe_gpu.mean() - oracle.force_errors(ref[tg], exact)["mean"]) <= 1e-9 * fe_gpu.mean()
    fb, tb = s.balance(x, y, z, m, *out)
    ofb, otb = oracle.balance(b.x, b.y, b.z, b.m, ref)
    assert fb <= 1e-14 and ofb <= 1e-14
    if variant == "UC":
        # the uncorrected torque imbalance is a property of the method, so
        # both sides see the same one
        assert abs(tb - otb) <= 1e-5 * otb and tb > 1e-10
    else:
        assert tb <= 1e-14 and otb <= 1e-14
    s.close()
