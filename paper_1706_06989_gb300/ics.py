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


def hernquist_disc(n: int, seed: int = 0, a: float = 1.0, disc_frac: float = 0.3,
                   h_r: float = 0.1, h_z: float = 0.01, rcut: float = 100.0) -> Bodies:
    """Hernquist halo (scale a, truncated at rcut * a) holding 1 - disc_frac of
    the mass, plus an exponential disc (surface density ~ exp(-R/h_r),
    sech^2 vertical profile of height h_z) holding disc_frac; equal masses."""
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
    m = np.full(n, 1.0 / n)
    return Bodies(x, y, z, m)


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
