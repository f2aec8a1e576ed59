"""The synthetic double white dwarf of Sec. 3's test problem (CPU): the
Lane-Emden integration against its closed-form solutions and tabulated
surface values, the Roche-lobe radius, the white-dwarf radius ratio, and the
sampled bodies against the polytropes' enclosed mass."""
import numpy as np
import pytest

from paper_1706_06989_gb300 import ics


def test_lane_emden_closed_forms():
    # n = 0: theta = 1 - xi^2/6, surface at sqrt(6), mass xi_1^3 / 3
    xi, th, m = ics.lane_emden(0.0)
    assert abs(xi[-1] - np.sqrt(6.0)) < 1e-9
    assert abs(m[-1] - np.sqrt(6.0) ** 3 / 3) < 1e-6
    assert np.allclose(th, 1 - xi ** 2 / 6, atol=1e-9)
    # n = 1: theta = sin(xi)/xi, surface at pi, mass pi
    xi, th, m = ics.lane_emden(1.0)
    assert abs(xi[-1] - np.pi) < 1e-9 and abs(m[-1] - np.pi) < 1e-6
    inner = slice(1, -1)
    assert np.allclose(th[inner], np.sin(xi[inner]) / xi[inner], atol=1e-10)
    # n = 5: theta = (1 + xi^2/3)^(-1/2), no surface; the mass tends to sqrt(3)
    xi, th, m = ics.lane_emden(5.0)
    assert np.allclose(th, (1 + xi ** 2 / 3) ** -0.5, atol=1e-9)
    x = xi[-1]
    assert abs(m[-1] - x ** 3 / 3 / (1 + x ** 2 / 3) ** 1.5) < 1e-6


@pytest.mark.parametrize("n,xi1,mass", [(1.5, 3.65375, 2.71406), (3.0, 6.89685, 2.01824)])
def test_lane_emden_tabulated_surfaces(n, xi1, mass):
    """The surface xi_1 and -xi_1^2 theta'(xi_1) of the two polytropes of the
    test problem, as tabulated (Chandrasekhar 1939) to five decimals."""
    xi, _, m = ics.lane_emden(n)
    assert abs(xi[-1] - xi1) < 1e-5 and abs(m[-1] - mass) < 1e-5


def test_roche_lobe_and_radius_ratio():
    # Eggleton (1983) at q = 1: 0.49 / (0.6 + ln 2)
    assert abs(ics.eggleton_roche_radius(1.0) - 0.49 / (0.6 + np.log(2.0))) < 1e-15
    # the lobe shrinks with the star's mass ratio
    assert ics.eggleton_roche_radius(0.2) < ics.eggleton_roche_radius(1.0)
    # cold white dwarfs shrink with mass; a Chandrasekhar-mass star has zero radius
    assert ics.wd_radius_ratio(1.0, 0.2) < 1.0
    assert ics.wd_radius_ratio(1.44, 0.2) == 0.0


def test_dwd_bodies_follow_the_polytropes():
    b = ics.dwd(200000, seed=1)
    mt = 1.2
    n_a = int(round(b.n / mt))
    assert b.n == 200000 and np.allclose(b.m, mt / b.n)
    p = b.pos()
    com = (b.m[:, None] * p).sum(0) / b.m.sum()
    assert np.abs(com).max() < 5e-3  # sampling noise of two finite stars
    ca, cd = np.array([-0.2 / mt, 0, 0]), np.array([1.0 / mt, 0, 0])
    ra = np.linalg.norm(p[:n_a] - ca, axis=1)
    rd = np.linalg.norm(p[n_a:] - cd, axis=1)
    r_don = ics.eggleton_roche_radius(0.2)
    r_acc = r_don * ics.wd_radius_ratio(1.0, 0.2)
    assert rd.max() <= r_don * (1 + 1e-12) and ra.max() <= r_acc * (1 + 1e-12)
    assert rd.max() > 0.95 * r_don  # the donor fills its lobe
    # enclosed-mass profile of each star against the Lane-Emden mass
    for r, R, n in ((ra, r_acc, 3.0), (rd, r_don, 1.5)):
        xi, _, m = ics.lane_emden(n)
        q = np.sort(r) / R * xi[-1]
        emp = np.arange(1, q.size + 1) / q.size
        model = np.interp(q, xi, m / m[-1])
        # Kolmogorov-Smirnov distance, below its 1% critical value
        assert np.abs(emp - model).max() < 1.63 / np.sqrt(q.size)
    # synchronous rotation about the centre of mass
    om = np.sqrt(mt)
    assert np.allclose(b.vx, -om * b.y) and np.allclose(b.vy, om * b.x) and np.all(b.vz == 0)
