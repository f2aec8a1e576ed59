"""a14: uniform kick-drift-kick leapfrog (Sec. 4: conservation needs uniform
steps), through the C ABI.

Parity: three steps against the same scheme written here with the oracle's
accelerations.  Conservation: with the torque-corrected variants the total
angular momentum stays at rounding level; the uncorrected variant drifts."""
import numpy as np
import pytest

import oracle
from paper_1706_06989_gb300 import ics

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state(b):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (b.x, b.y, b.z, b.vx, b.vy, b.vz, b.m)]


def _solver(**kw):
    from paper_1706_06989_gb300 import fmm
    return fmm.FMM(**kw)


def test_leapfrog_matches_oracle_integration():
    b = ics.binary_plummer(3000, seed=3)
    dt = 2 * np.pi / np.sqrt(1.5) / 1000
    st = _state(b)
    s = _solver(theta=0.5, variant="TC")
    s.leapfrog(*st, dt=dt, nsteps=3)
    gx = torch.stack(st[:3], 1).cpu().numpy()
    gv = torch.stack(st[3:6], 1).cpu().numpy()
    # the same steps on the CPU: v += a dt/2, x += v dt, a = a(x), v += a dt/2
    x, v, m = b.pos().copy(), np.stack([b.vx, b.vy, b.vz], 1).copy(), b.m

    def acc(p):
        return oracle.Oracle(p[:, 0], p[:, 1], p[:, 2], m, 0.5, 25).accel("TC")

    a = acc(x)
    for _ in range(3):
        v += 0.5 * dt * a
        x += dt * v
        a = acc(x)
        v += 0.5 * dt * a
    assert np.abs(gx - x).max() <= 1e-12 * np.abs(x).max()
    assert np.abs(gv - v).max() <= 1e-10 * np.abs(v).max()


@pytest.mark.parametrize("variant", ["TC", "TCO"])
def test_leapfrog_conserves_momenta(variant):
    b = ics.binary_plummer(20000, seed=4)
    dt = 2 * np.pi / np.sqrt(1.5) / 1000
    st = _state(b)
    s = _solver(theta=0.5, variant=variant)
    _, mom = s.leapfrog(*st, dt=dt, nsteps=20)
    mom = mom.cpu().numpy()
    m = b.m
    p_scale = np.sum(m * np.sqrt(b.vx ** 2 + b.vy ** 2 + b.vz ** 2))
    l_scale = np.sum(m * np.linalg.norm(np.cross(b.pos(), np.stack([b.vx, b.vy, b.vz], 1)), axis=1))
    dp = np.abs(mom[1:, :3] - mom[:-1, :3]).max() / p_scale
    dl = np.abs(mom[1:, 3:] - mom[:-1, 3:]).max() / l_scale
    assert dp <= 1e-15, dp
    assert dl <= 1e-14, dl


def test_uncorrected_variant_drifts_in_angular_momentum():
    b = ics.binary_plummer(20000, seed=4)
    dt = 2 * np.pi / np.sqrt(1.5) / 1000
    drift = {}
    for v in ("UC", "TC"):
        st = _state(b)
        _, mom = _solver(theta=0.5, variant=v).leapfrog(*st, dt=dt, nsteps=20)
        mom = mom.cpu().numpy()
        drift[v] = np.abs(mom[-1, 3:] - mom[0, 3:]).max()
    assert drift["UC"] > 100 * drift["TC"], drift


def test_softened_leapfrog_matches_oracle_integration():
    """The same three steps with Plummer softening (the oracle's softened
    accelerations), and the torque-corrected variant still conserving the
    angular momentum at rounding."""
    b = ics.binary_plummer(3000, seed=5)
    dt = 2 * np.pi / np.sqrt(1.5) / 1000
    eps = 0.01
    st = _state(b)
    s = _solver(theta=0.5, variant="TC")
    s.set_softening(eps)
    _, mom = s.leapfrog(*st, dt=dt, nsteps=3)
    gx = torch.stack(st[:3], 1).cpu().numpy()
    gv = torch.stack(st[3:6], 1).cpu().numpy()
    x, v, m = b.pos().copy(), np.stack([b.vx, b.vy, b.vz], 1).copy(), b.m

    def acc(p):
        return oracle.Oracle(p[:, 0], p[:, 1], p[:, 2], m, 0.5, 25, softening=eps).accel("TC")

    a = acc(x)
    for _ in range(3):
        v += 0.5 * dt * a
        x += dt * v
        a = acc(x)
        v += 0.5 * dt * a
    assert np.abs(gx - x).max() <= 1e-12 * np.abs(x).max()
    assert np.abs(gv - v).max() <= 1e-10 * np.abs(v).max()
    mom = mom.cpu().numpy()
    l_scale = np.sum(m * np.linalg.norm(np.cross(b.pos(), np.stack([b.vx, b.vy, b.vz], 1)), axis=1))
    assert np.abs(mom[1:, 3:] - mom[:-1, 3:]).max() / l_scale <= 1e-14
