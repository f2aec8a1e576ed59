"""CPU models of two pieces of kernel arithmetic, checked exactly.

1. The FP64 near field's pair factor r^-3 (csrc/p2p.cu, inv_r3): a 24-bit
   seed y0 ~ r^-1 from an FP32 reciprocal square root of the leading bits of
   r^2 = m 4^k, moved between formats by integer operations on the bit
   patterns, then r^-3 = y0^3 (1 - e)^(-3/2) with e = 1 - r^2 y0^2 and the
   binomial series taken to second order.  The model replays those steps with
   exact rational arithmetic standing in for each FMA's single rounding, and
   with seeds off by a few FP32 units (a hardware reciprocal square root is
   an approximation), and bounds the relative error against the exact value.

2. The FP64 order-3 M2L reduction's lane plan (csrc/m2l.cu, k_m2l_reduce):
   24-double slots read as one flat array, 32 values per load; a U2 or U3
   value is scaled by its slot's factor, which one shuffle per load brings
   from the lane that loaded it (that lane's own value, or its value of the
   next load).  The model runs the same bookkeeping and compares with the
   direct per-slot sums.
"""
import math
import struct
from fractions import Fraction

import numpy as np


def _d2b(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _b2d(b):
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _f2u(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _u2f(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _inv_r3_model(r2, seed_ulps=0):
    bits = _d2b(r2)
    E = (bits >> 52) - 1023
    k = E >> 1
    mf = ((E - 2 * k + 127) << 23) | ((bits >> 29) & 0x7FFFFF)
    m = _u2f(mf)
    assert 1.0 <= m < 4.0
    yf = _f2u(float(np.float32(1.0 / math.sqrt(m)))) + seed_ulps
    y0 = _b2d((((yf >> 23) - 127 + 1023 - k) << 52) | ((yf & 0x7FFFFF) << 29))
    y2 = y0 * y0
    assert Fraction(y2) == Fraction(y0) ** 2  # a 24-bit y0 squares exactly
    e = _fma(-r2, y2, 1.0)
    y3 = y2 * y0
    return _fma(y3, e * _fma(e, 1.875, 1.5), y3)


def _exact_inv_r3(r2):
    # r^-3 = 1 / (r^2 sqrt(r^2)), the root to about 600 bits by an integer square root
    f = Fraction(r2)
    s = Fraction(math.isqrt(math.floor(f * 2 ** 2000)), 2 ** 1000)
    return 1 / (f * s)


def test_near_field_inv_r3_model_error_bound():
    rng = np.random.default_rng(3)
    worst = 0.0
    r2s = list(10.0 ** rng.uniform(-200, 200, 600)) + list(rng.uniform(1e-6, 100, 300))
    r2s += [1.0, 2.0, 4.0, 3.999999999999999, np.nextafter(1.0, 2.0), 2.0 ** -601, 2.0 ** 600]
    for r2 in r2s:
        r2 = float(r2)
        ref = _exact_inv_r3(r2)
        for u in (-4, 0, 4):
            got = _inv_r3_model(r2, u)
            worst = max(worst, float(abs(Fraction(got) - ref) / ref) / 2.0 ** -53)
    # two roundings (y0^3 and the final FMA) plus the omitted e^3 term
    assert worst <= 3.0, worst


def _red_sends_next(u, t, S=24, phases=3):
    p = 32 * (u + 1) + t
    r = p % S
    first = p - r + (3 if r == 19 else 9)
    return u + 1 < phases and r in (19, 20) and first < 32 * (u + 1)


def _scale_off(q):
    return 19 - q if q < 9 else 20 - q


def _reduce_model(flat, S=24, phases=3, periods=2):
    e1 = len(flat)
    acc = np.zeros((32, phases))
    for b in range(0, e1, periods * phases * 32):
        for h in range(periods):
            v = np.zeros((32, phases))
            for l in range(32):
                for u in range(phases):
                    e = b + l + 32 * (h * phases + u)
                    v[l, u] = flat[e] if e < e1 else 0.0
            for u in range(phases):
                send = [v[t, u + 1] if _red_sends_next(u, t) else v[t, u] for t in range(32)]
                for l in range(32):
                    q = (l + 32 * u) % S
                    f = send[(l + _scale_off(q)) & 31]
                    if b + l + 32 * (h * phases + u) < e1:
                        acc[l, u] += v[l, u] * (1.0 if q < 3 else f)
    loc = np.zeros(19)
    for q in range(19):
        for u in range(phases):
            r = (q - 32 * u) % S
            loc[q] += acc[r, u]
            if r + S < 32:
                loc[q] += acc[r + S, u]
    return loc


def test_m2l_reduce_lane_plan_model():
    rng = np.random.default_rng(5)
    for nslot in (0, 1, 3, 4, 5, 7, 8, 9, 31, 33, 57):
        sl = rng.normal(size=(nslot, 24))
        sl[:, 21:] = rng.normal(size=(nslot, 3)) * 1e30  # pad: never read into a coefficient
        got = _reduce_model(sl.ravel())
        ref = np.concatenate([sl[:, :3].sum(0), (sl[:, 3:9] * sl[:, 19:20]).sum(0),
                              (sl[:, 9:19] * sl[:, 20:21]).sum(0)]) if nslot else np.zeros(19)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), nslot
