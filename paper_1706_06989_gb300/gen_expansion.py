"""Generates csrc/expansion_gen.cuh: straight-line CUDA for the general-order
Cartesian expansion of App. A (orders P = 4 and 5), in multi-index form.

Notation (alpha, beta, gamma are exponent triples; |a| their order; a! the
product of factorials):
  moments      M^a   = sum mu x^a about the centre of mass (Eqs. 1-3, App. A)
  derivatives  D^g   = d^g G(r), G = -1/R, written D^g = R^-(|g|+1) U^g(n) with
               n = r/R and U^g a polynomial in n (chain rule on G(u), u = r.r:
               every derivative pairs some of its indices through u's second
               derivative and leaves the others as components of r)
  field of B at A:  L_A^a = sum_b (-1)^|b| D^(a+b) M_B^b / b!,  |a| + |b| <= P
  field of A at B:  L_B^b = (-1)^|b| sum_a D^(a+b) M_A^a / a!
  body at x:        g_k = - sum_a L^(a+e_k) x^a / a!,  |a| <= P - 1
  correction:       F_k = - sum_{|a|+|b|=P} (-1)^|b| M_A^a M_B^b D^(a+b+e_k)/(a! b!)
                    applied as +F/M_A on A and -F/M_B on B; the alternative
                    F' = F - n (n.F) removes its component along r.
  M2M: M^a(parent) = sum_{b <= a} C(a, b) M^b(child) s^(a-b), s = Z_child - Z
  L2L: L'^a = sum_g L^(a+g) s^g / g!
Moments are scaled as M^b R^-|b| before the contractions, so that no large
power of 1/R is formed on its own.

Run `python gen_expansion.py` to rewrite csrc/expansion_gen.cuh; the build
uses the committed header.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

ORDERS = (4, 5)
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "expansion_gen.cuh")


def multi(n):
    """Exponent triples of order n: a = n..0, then b = n-a..0."""
    return [(a, b, n - a - b) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


def all_multi(P):
    out = []
    for n in range(P + 1):
        out += multi(n)
    return out


def idx_table(P):
    return {m: i for i, m in enumerate(all_multi(P))}


def fact(t):
    return math.factorial(t[0]) * math.factorial(t[1]) * math.factorial(t[2])


def add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def lit(x) -> str:
    """A C++ literal of type T for a rational."""
    x = Fraction(x)
    if x.denominator == 1:
        return f"T({x.numerator})"
    return f"T({float(x)!r})"


def dfact(k):
    """(2m - 1)!! with (-1)!! = 1."""
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def u_terms(g):
    """U^g(n) = sum coef * nx^p ny^q nz^s, from the pairing of equal indices."""
    a, b, c = g
    n = a + b + c
    terms = []
    for i in range(a // 2 + 1):
        for j in range(b // 2 + 1):
            for l in range(c // 2 + 1):
                m = n - i - j - l
                cm = -((-1) ** m) * dfact(2 * m - 1)
                k = (math.factorial(a) // (2 ** i * math.factorial(i) * math.factorial(a - 2 * i))) * \
                    (math.factorial(b) // (2 ** j * math.factorial(j) * math.factorial(b - 2 * j))) * \
                    (math.factorial(c) // (2 ** l * math.factorial(l) * math.factorial(c - 2 * l)))
                terms.append((cm * k, a - 2 * i, b - 2 * j, c - 2 * l))
    return terms


def emit_P(P: int) -> str:
    NM = (P + 1) * (P + 2) * (P + 3) // 6
    NU = (P + 2) * (P + 3) * (P + 4) // 6
    mi = all_multi(P)
    mu = all_multi(P + 1)
    im = idx_table(P)
    iu = idx_table(P + 1)
    L = []
    w = L.append
    w(f"// ---------------- order P = {P}: {NM} moments, {NM - 1} local coefficients ----------------")
    w(f"template <> struct Expansion<{P}> {{")
    w(f"  static constexpr int kNM = {NM};  // moments of order 0..P")
    w(f"  static constexpr int kNL = {NM - 1};  // local coefficients of order 1..P")
    # ---- U^g(n) for |g| <= P + 1
    w("  template <class T>")
    w("  __device__ static __forceinline__ void unit_derivs(T nx, T ny, T nz, T *U) {")
    w(f"    T px[{P + 2}], py[{P + 2}], pz[{P + 2}];")
    w("    px[0] = py[0] = pz[0] = T(1);")
    w(f"#pragma unroll\n    for (int k = 1; k <= {P + 1}; ++k) {{ px[k] = px[k - 1] * nx; py[k] = py[k - 1] * ny; pz[k] = pz[k - 1] * nz; }}")
    for g in mu:
        terms = u_terms(g)
        expr = " + ".join(f"{lit(cf)} * (px[{p}] * py[{q}] * pz[{s}])" for cf, p, q, s in terms)
        w(f"    U[{iu[g]}] = {expr};")
    w("  }")
    # ---- M2L for one pair: A side and B side locals, correction
    w("  // one accepted pair: locals of A (field of B) and of B (field of A)")
    w("  template <class T, int VARIANT>")
    w("  __device__ static __forceinline__ void m2l(const T r[3], const T *mA, const T *mB, T iMA, T iMB,")
    w("                                            T *LA, T *LB, T min_r2) {")
    w("    const T R2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];")
    w("    if (!(R2 > min_r2)) {")
    w(f"#pragma unroll\n      for (int q = 0; q < {NM - 1}; ++q) LA[q] = LB[q] = T(0);")
    w("      return;")
    w("    }")
    w("    const T Ri = rsqrt_t(R2);")
    w("    const T nx = r[0] * Ri, ny = r[1] * Ri, nz = r[2] * Ri;")
    w(f"    T ri[{P + 3}];")
    w(f"    ri[0] = T(1);\n#pragma unroll\n    for (int k = 1; k <= {P + 2}; ++k) ri[k] = ri[k - 1] * Ri;")
    w(f"    T U[{NU}];")
    w("    unit_derivs<T>(nx, ny, nz, U);")
    w(f"    T sA[{NM}], sB[{NM}];")
    for i, m in enumerate(mi):
        o = sum(m)
        w(f"    sA[{i}] = mA[{i}] * ri[{o}]; sB[{i}] = mB[{i}] * ri[{o}];")
    # A side
    for a in mi:
        if sum(a) == 0:
            continue
        terms = []
        for b in mi:
            if sum(a) + sum(b) > P:
                continue
            cf = Fraction((-1) ** sum(b), fact(b))
            terms.append(f"{lit(cf)} * U[{iu[add(a, b)]}] * sB[{im[b]}]")
        w(f"    LA[{im[a] - 1}] = ri[{sum(a) + 1}] * ({' + '.join(terms)});")
    # B side
    for b in mi:
        if sum(b) == 0:
            continue
        terms = []
        for a in mi:
            if sum(a) + sum(b) > P:
                continue
            cf = Fraction(1, fact(a))
            terms.append(f"{lit(cf)} * U[{iu[add(a, b)]}] * sA[{im[a]}]")
        sgn = "" if sum(b) % 2 == 0 else "-"
        w(f"    LB[{im[b] - 1}] = {sgn}ri[{sum(b) + 1}] * ({' + '.join(terms)});")
    # correction
    w("    if (VARIANT != FMM_UC) {")
    for k, e in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        terms = []
        for a in mi:
            for b in mi:
                if sum(a) + sum(b) != P:
                    continue
                cf = Fraction(-((-1) ** sum(b)), fact(a) * fact(b))
                terms.append(f"{lit(cf)} * sA[{im[a]}] * sB[{im[b]}] * U[{iu[add(add(a, b), e)]}]")
        w(f"      T F{k} = ri[2] * ({' + '.join(terms)});")
    w("      if (VARIANT == FMM_TCO) {")
    w("        const T nf = nx * F0 + ny * F1 + nz * F2;")
    w("        F0 -= nx * nf; F1 -= ny * nf; F2 -= nz * nf;")
    w("      }")
    w("      LA[0] -= F0 * iMA; LA[1] -= F1 * iMA; LA[2] -= F2 * iMA;")
    w("      LB[0] += F0 * iMB; LB[1] += F1 * iMB; LB[2] += F2 * iMB;")
    w("    }")
    w("  }")
    # ---- P2M: add one body's moments
    w("  __device__ static __forceinline__ void p2m_add(double *mo, double mu, double x, double y, double z) {")
    w(f"    double px[{P + 1}], py[{P + 1}], pz[{P + 1}];")
    w("    px[0] = py[0] = pz[0] = 1.0;")
    w(f"#pragma unroll\n    for (int k = 1; k <= {P}; ++k) {{ px[k] = px[k - 1] * x; py[k] = py[k - 1] * y; pz[k] = pz[k - 1] * z; }}")
    for i, (a, b, c) in enumerate(mi):
        w(f"    mo[{i}] += mu * (px[{a}] * py[{b}] * pz[{c}]);")
    w("  }")
    # ---- M2M: add a child's shifted moments
    w("  __device__ static __forceinline__ void m2m_add(double *mp, const double *mc, const double s[3]) {")
    w(f"    double px[{P + 1}], py[{P + 1}], pz[{P + 1}];")
    w("    px[0] = py[0] = pz[0] = 1.0;")
    w(f"#pragma unroll\n    for (int k = 1; k <= {P}; ++k) {{ px[k] = px[k - 1] * s[0]; py[k] = py[k - 1] * s[1]; pz[k] = pz[k - 1] * s[2]; }}")
    for a in mi:
        terms = []
        for b in mi:
            if b[0] <= a[0] and b[1] <= a[1] and b[2] <= a[2]:
                cf = math.comb(a[0], b[0]) * math.comb(a[1], b[1]) * math.comb(a[2], b[2])
                d = (a[0] - b[0], a[1] - b[1], a[2] - b[2])
                mono = f"px[{d[0]}] * py[{d[1]}] * pz[{d[2]}]"
                terms.append(f"{float(cf)!r} * mc[{im[b]}] * ({mono})")
        w(f"    mp[{im[a]}] += {' + '.join(terms)};")
    w("  }")
    # ---- L2L: parent's locals shifted by s, added to the child's
    w("  __device__ static __forceinline__ void l2l_add(double *Lc, const double *Lp, const double s[3]) {")
    w(f"    double px[{P + 1}], py[{P + 1}], pz[{P + 1}];")
    w("    px[0] = py[0] = pz[0] = 1.0;")
    w(f"#pragma unroll\n    for (int k = 1; k <= {P}; ++k) {{ px[k] = px[k - 1] * s[0]; py[k] = py[k - 1] * s[1]; pz[k] = pz[k - 1] * s[2]; }}")
    for a in mi:
        if sum(a) == 0:
            continue
        terms = []
        for g in mi:
            ag = add(a, g)
            if sum(ag) > P:
                continue
            cf = Fraction(1, fact(g))
            mono = f"px[{g[0]}] * py[{g[1]}] * pz[{g[2]}]"
            terms.append(f"{float(cf)!r} * Lp[{im[ag] - 1}] * ({mono})")
        w(f"    Lc[{im[a] - 1}] += {' + '.join(terms)};")
    w("  }")
    # ---- L2P: acceleration at offset x
    w("  __device__ static __forceinline__ void l2p(const double *Lc, const double x[3], double g[3]) {")
    w(f"    double px[{P}], py[{P}], pz[{P}];")
    w("    px[0] = py[0] = pz[0] = 1.0;")
    w(f"#pragma unroll\n    for (int k = 1; k < {P}; ++k) {{ px[k] = px[k - 1] * x[0]; py[k] = py[k - 1] * x[1]; pz[k] = pz[k - 1] * x[2]; }}")
    for k, e in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        terms = []
        for a in mi:
            if sum(a) > P - 1:
                continue
            cf = Fraction(1, fact(a))
            mono = f"px[{a[0]}] * py[{a[1]}] * pz[{a[2]}]"
            terms.append(f"{float(cf)!r} * Lc[{im[add(a, e)] - 1}] * ({mono})")
        w(f"    g[{k}] = -({' + '.join(terms)});")
    w("  }")
    w("};")
    return "\n".join(L)


def render() -> str:
    parts = ["// expansion_gen.cuh -- GENERATED by gen_expansion.py; do not edit.",
             "// General-order Cartesian expansion of App. A in multi-index form (see the",
             "// generator's docstring for the formulas).  Included by expansion.cu.",
             "#pragma once",
             "",
             "template <int P> struct Expansion;",
             ""]
    for P in ORDERS:
        parts.append(emit_P(P))
        parts.append("")
    return "\n".join(parts) + "\n"


def main():
    with open(OUT, "w") as f:
        f.write(render())
    print(OUT)


if __name__ == "__main__":
    main()
