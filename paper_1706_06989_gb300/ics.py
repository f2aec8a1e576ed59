"""Seeded synthetic inputs (initial conditions) shared by the tests, the bench
and the CPU oracle's callers.

This module draws bodies and nothing else: it holds none of the method's
arithmetic.  Every generator uses ``numpy.random.Generator(PCG64(seed))`` and
returns structure-of-arrays float64 data (x, y, z, m[, vx, vy, vz]) with G = 1.

The paper's own test problem (a double white dwarf of two Lane-Emden
polytropes, Sec. 3) is replaced by Plummer spheres, a binary of two Plummer
spheres, a Hernquist halo with an exponential disc, and ensembles of Plummer
spheres of log-uniform size.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np


@dataclass
class Bodies:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray
    vx: np.ndarray | None = None
    vy: np.ndarray | None = None
    vz: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def pos(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _directions(rng: np.random.Generator, n: int) -> np.ndarray:
    cz = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(1.0 - cz * cz)
    return np.stack([s * np.cos(phi), s * np.sin(phi), cz], axis=1)


def _plummer_radii(rng: np.random.Generator, n: int, a: float, rcut: float) -> np.ndarray:
    """Radii from the inverse cumulative mass of a Plummer sphere
    (Aarseth, Henon & Wielen 1974), redrawing radii beyond rcut."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        k = n - filled
        X = rng.uniform(0.0, 1.0, k)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        ok = np.isfinite(r) & (r <= rcut)
        good = r[ok]
        out[filled:filled + good.shape[0]] = good
        filled += good.shape[0]
    return out


def _plummer_speeds(rng: np.random.Generator, r: np.ndarray, M: float, a: float) -> np.ndarray:
    """Isotropic equilibrium speeds: q = v / v_esc drawn from q^2 (1-q^2)^(7/2)
    by rejection (Aarseth, Henon & Wielen 1974)."""
    n = r.shape[0]
    q = np.empty(n)
    filled = 0
    while filled < n:
        k = 2 * (n - filled) + 16
        x = rng.uniform(0.0, 1.0, k)
        y = rng.uniform(0.0, 0.1, k)
        g = x * x * (1.0 - x * x) ** 3.5
        acc = x[y < g]
        take = min(acc.shape[0], n - filled)
        q[filled:filled + take] = acc[:take]
        filled += take
    vesc = np.sqrt(2.0 * M / a) * (1.0 + (r / a) ** 2) ** -0.25
    return q * vesc


def plummer(n: int, seed: int = 0, M: float = 1.0, a: float = 1.0, rcut: float = 20.0,
            velocities: bool = False) -> Bodies:
    """Plummer sphere of n equal-mass bodies, total mass M, scale radius a,
    truncated at rcut * a."""
    rng = _rng(seed)
    r = _plummer_radii(rng, n, a, rcut * a)
    pos = r[:, None] * _directions(rng, n)
    m = np.full(n, M / n)
    b = Bodies(pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(), m)
    if velocities:
        v = _plummer_speeds(rng, r, M, a)[:, None] * _directions(rng, n)
        b.vx, b.vy, b.vz = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    return b


def binary_plummer(n: int, seed: int = 0, m1: float = 0.6, a1: float = 0.05, m2: float = 0.9,
                   a2: float = 0.04, sep: float = 1.0) -> Bodies:
    """Two Plummer spheres on a circular orbit about their common centre of
    mass, equal-mass bodies split by mass, each sphere with its own isotropic
    equilibrium velocities added to the orbital velocity."""
    mt = m1 + m2
    n1 = int(round(n * m1 / mt))
    n2 = n - n1
    s1 = plummer(n1, seed=2 * seed + 11, M=m1, a=a1, velocities=True)
    s2 = plummer(n2, seed=2 * seed + 12, M=m2, a=a2, velocities=True)
    omega = np.sqrt(mt / sep ** 3)
    c1 = -sep * m2 / mt
    c2 = sep * m1 / mt
    x = np.concatenate([s1.x + c1, s2.x + c2])
    y = np.concatenate([s1.y, s2.y])
    z = np.concatenate([s1.z, s2.z])
    vx = np.concatenate([s1.vx, s2.vx])
    vy = np.concatenate([s1.vy + omega * c1, s2.vy + omega * c2])
    vz = np.concatenate([s1.vz, s2.vz])
    m = np.full(n, mt / n)
    return Bodies(x, y, z, m, vx, vy, vz)


def power_law_masses(rng: np.random.Generator, n: int, total: float, slope: float = 2.35,
                     ratio: float = 100.0) -> np.ndarray:
    """n masses drawn from dN/dm ~ m^-slope on [1, ratio] (inverse cumulative
    distribution; slope 2.35 is Salpeter's), scaled to sum to total."""
    u = rng.uniform(0.0, 1.0, n)
    e = 1.0 - slope
    m = (1.0 + u * (ratio ** e - 1.0)) ** (1.0 / e)
    return m * (total / m.sum())


def hernquist_disc(n: int, seed: int = 0, a: float = 1.0, disc_frac: float = 0.3,
                   h_r: float = 0.1, h_z: float = 0.01, rcut: float = 100.0,
                   mass_spectrum: bool = False) -> Bodies:
    """Hernquist halo (scale a, truncated at rcut * a) holding 1 - disc_frac of
    the mass, plus an exponential disc (surface density ~ exp(-R/h_r),
    sech^2 vertical profile of height h_z) holding disc_frac; equal masses,
    or (mass_spectrum) masses over two decades from a Salpeter power law,
    each component keeping its share of the mass."""
    rng = _rng(seed)
    nd = int(round(n * disc_frac))
    nh = n - nd
    r = np.empty(nh)
    filled = 0
    while filled < nh:
        k = nh - filled
        s = np.sqrt(rng.uniform(0.0, 1.0, k))
        with np.errstate(divide="ignore"):
            rr = a * s / (1.0 - s)
        good = rr[np.isfinite(rr) & (rr <= rcut * a)]
        r[filled:filled + good.shape[0]] = good
        filled += good.shape[0]
    ph = r[:, None] * _directions(rng, nh)
    R = h_r * rng.gamma(2.0, 1.0, nd)
    phi = rng.uniform(0.0, 2.0 * np.pi, nd)
    u = rng.uniform(0.0, 1.0, nd)
    u = np.clip(u, 1e-15, 1.0 - 1e-15)
    zd = h_z * np.arctanh(2.0 * u - 1.0)
    x = np.concatenate([ph[:, 0], R * np.cos(phi)])
    y = np.concatenate([ph[:, 1], R * np.sin(phi)])
    z = np.concatenate([ph[:, 2], zd])
    if mass_spectrum:
        m = np.concatenate([power_law_masses(rng, nh, 1.0 - disc_frac), power_law_masses(rng, nd, disc_frac)])
    else:
        m = np.full(n, 1.0 / n)
    return Bodies(x, y, z, m)


@functools.lru_cache(maxsize=16)
def lane_emden(n_index: float, h: float = 1e-3):
    """Lane-Emden polytrope of index n: theta'' + (2/xi) theta' + theta^n = 0,
    theta(0) = 1, theta'(0) = 0, integrated by classical fourth-order
    Runge-Kutta in xi from a series start (theta = 1 - xi^2/6 + n xi^4/120)
    to the first zero xi_1 (the stellar surface), which is located by a final
    step to the zero of the cubic Hermite interpolant.  Returns (xi, theta,
    mass) on the grid, mass = -xi^2 theta' (the mass inside xi in units of
    4 pi rho_c alpha^3), with xi[-1] = xi_1.  For n >= 5 there is no zero;
    the integration then stops at xi = 50."""
    def rhs(x, y):
        t, dt = y
        # theta^n with theta clipped at the surface (the stages of the last
        # step may step past the zero)
        return np.array([dt, -max(t, 0.0) ** n_index - 2.0 * dt / x])

    x0 = 1e-3
    xs = [0.0, x0]
    ts = [1.0, 1.0 - x0 ** 2 / 6 + n_index * x0 ** 4 / 120]
    ds = [0.0, -x0 / 3 + n_index * x0 ** 3 / 30]
    y = np.array([ts[-1], ds[-1]])
    x = x0
    while x < 50.0:
        k1 = rhs(x, y)
        k2 = rhs(x + h / 2, y + h / 2 * k1)
        k3 = rhs(x + h / 2, y + h / 2 * k2)
        k4 = rhs(x + h, y + h * k3)
        yn = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if yn[0] <= 0.0:
            # zero of the cubic Hermite interpolant on [x, x + h]
            lo, hi = 0.0, 1.0
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                s2, s3 = mid * mid, mid * mid * mid
                val = ((2 * s3 - 3 * s2 + 1) * y[0] + (s3 - 2 * s2 + mid) * h * y[1]
                       + (-2 * s3 + 3 * s2) * yn[0] + (s3 - s2) * h * yn[1])
                lo, hi = (mid, hi) if val > 0 else (lo, mid)
            tz = 0.5 * (lo + hi)
            xz = x + tz * h
            dz = y[1] + tz * (yn[1] - y[1])  # theta' varies slowly over one step
            xs.append(xz)
            ts.append(0.0)
            ds.append(dz)
            break
        x += h
        y = yn
        xs.append(x)
        ts.append(y[0])
        ds.append(y[1])
    xi, th, dth = np.array(xs), np.array(ts), np.array(ds)
    return xi, th, -xi * xi * dth


def _polytrope_radii(rng: np.random.Generator, n: int, n_index: float, radius: float) -> np.ndarray:
    """Radii of n bodies sampling a Lane-Emden polytrope of the given index
    and surface radius: the inverse of the normalised enclosed mass."""
    xi, _, mass = lane_emden(n_index)
    cdf = mass / mass[-1]
    cdf, keep = np.unique(cdf, return_index=True)
    u = rng.uniform(0.0, 1.0, n)
    return radius * np.interp(u, cdf, xi[keep]) / xi[-1]


def eggleton_roche_radius(q: float) -> float:
    """Volume-equivalent Roche-lobe radius over the separation for a star of
    mass ratio q = M_star / M_companion (Eggleton 1983)."""
    q23 = q ** (2.0 / 3.0)
    return 0.49 * q23 / (0.6 * q23 + np.log1p(q ** (1.0 / 3.0)))


def wd_radius_ratio(m1: float, m2: float, m_ch: float = 1.44) -> float:
    """R(m1) / R(m2) of cold white dwarfs by the Nauenberg (1972) mass-radius
    relation R ~ [(M/M_ch)^(-2/3) - (M/M_ch)^(2/3)]^(1/2)."""
    f = lambda m: np.sqrt((m / m_ch) ** (-2.0 / 3.0) - (m / m_ch) ** (2.0 / 3.0))
    return float(f(m1) / f(m2))


def dwd(n: int, seed: int = 0, m_acc: float = 1.0, m_don: float = 0.2, n_acc: float = 3.0,
        n_don: float = 1.5, sep: float = 1.0) -> Bodies:
    """The test problem of Sec. 3 as synthetic bodies: a double white dwarf of
    an accretor (mass 1, Lane-Emden index 3) and a donor (mass 0.2, index 1.5)
    that fills its Roche lobe, each star spherical, n equal-mass bodies split
    by mass and sampled from the polytropes' densities.  Readings of what the
    paper leaves open: the separation is the unit of length (sep = 1); the
    donor's radius is the volume-equivalent Roche-lobe radius (Eggleton 1983)
    at q = m_don / m_acc; the accretor's radius follows from the donor's by
    the cold white-dwarf mass-radius relation (Nauenberg 1972).  Masses in
    solar masses with G = 1.  The stars sit on the x axis about the common
    centre of mass and rotate rigidly with the orbit (velocities
    Omega z x X, Omega = sqrt(M / sep^3))."""
    rng = _rng(seed)
    mt = m_acc + m_don
    n_a = int(round(n * m_acc / mt))
    n_d = n - n_a
    r_don = eggleton_roche_radius(m_don / m_acc) * sep
    r_acc = r_don * wd_radius_ratio(m_acc, m_don)
    pa = _polytrope_radii(rng, n_a, n_acc, r_acc)[:, None] * _directions(rng, n_a)
    pd = _polytrope_radii(rng, n_d, n_don, r_don)[:, None] * _directions(rng, n_d)
    pa[:, 0] += -sep * m_don / mt
    pd[:, 0] += sep * m_acc / mt
    p = np.concatenate([pa, pd])
    omega = np.sqrt(mt / sep ** 3)
    m = np.full(n, mt / n)
    return Bodies(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m,
                  -omega * p[:, 1], omega * p[:, 0], np.zeros(n))


def ensemble_sizes(nsys: int = 512, seed: int = 0, nmin: int = 1024, nmax: int = 65536) -> np.ndarray:
    """Sizes drawn log-uniformly in [nmin, nmax]."""
    rng = _rng(seed)
    u = rng.uniform(np.log(nmin), np.log(nmax), nsys)
    return np.minimum(np.floor(np.exp(u)).astype(np.int64), nmax)


def ensemble(nsys: int = 512, seed: int = 0, nmin: int = 1024, nmax: int = 65536):
    """Independent Plummer spheres (seed per system); returns (offsets, Bodies)."""
    sizes = ensemble_sizes(nsys, seed, nmin, nmax)
    parts = [plummer(int(s), seed=1000 + k) for k, s in enumerate(sizes)]
    offsets = np.zeros(nsys + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    cat = lambda f: np.concatenate([getattr(p, f) for p in parts])
    return offsets, Bodies(cat("x"), cat("y"), cat("z"), cat("m"))


def error_subset(n: int, k: int = 4096, seed: int = 1) -> np.ndarray:
    """k distinct body indices (all of them when n <= k), sorted."""
    if n <= k:
        return np.arange(n, dtype=np.int64)
    return np.sort(_rng(seed).choice(n, size=k, replace=False)).astype(np.int64)


def uniform_cube(n: int, seed: int = 0, mass_spread: bool = False) -> Bodies:
    """Uniform random bodies in the unit cube (edge cases and small tests);
    optionally with masses spread over a decade."""
    rng = _rng(seed)
    p = rng.uniform(0.0, 1.0, (n, 3))
    m = rng.uniform(0.1, 1.0, n) if mass_spread else np.full(n, 1.0 / n)
    return Bodies(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m)
