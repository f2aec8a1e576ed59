"""Oracle of the dual-tree walk with the learned pair selector (test
infrastructure only; the product library never imports it).

Sec. 2 lets any pair selection driven by an error estimate replace the fixed
opening angle, as long as every accepted pair still interacts mutually.  The
GPU path uses a small network as that estimate, inside a band: the opening
criterion at theta keeps accepting what it accepts; a pair that it rejects
but that the criterion at theta_max <= 1 accepts (theta_max = 1 is the safety
bound |Z_A - Z_B| >= R_A + R_B, the loosest angle Sec. 2 allows), and that
holds at least ``min_work`` body pairs, is scored, and accepted when

    score = pred + adj < log10_target,

with ``pred`` the network's predicted log10 error of the pair in units of the
partner's monopole field M/|r|^2 (the worse side), and

    absolute rule:  adj = log10 max(M_A, M_B) - 2 log10 |r|
    relative rule:  adj = log10 max(M_B / (|r|^2 |a_A|), M_A / (|r|^2 |a_B|)),

|a_c| an estimate of the field at cell c (below).  Every other pair follows
the walk of Sec. 2: leaf pairs are summed directly, otherwise one cell is
opened.

This module restates that walk in plain numpy over the C oracle's tree
(``oracle.Oracle``): features from the oracle's FP64 geometry, the network
through ``oracle.mlp.forward(..., "bf16")``, the criterion as the oracle
evaluates it (theta^2 d^2 >= (R_A + R_B)^2, no FMA, equality accepted).  The
walk is breadth first, which gives the same pair set as any other order: the
set depends only on the decision taken for each pair.

Features of a pair (the pair is first ordered by R_max rounded to FP32,
descending, then by cell id, so that (A, B) and (B, A) agree): log10 |r|,
log10 R_A/|r| and log10 R_B/|r| (each floored at -12), log10 M_A,
log10 M_B, log10 of (|Q - tr(Q)/3 I|_F / (M R_max^2) + 1e-12) of A and of B
(the norm taken as 0 for a cell of one body or of zero extent), and
log10 (N_A + N_B).

The field estimate of the relative rule: the monopoles of one coarse level
of the tree (the deepest level before the first level with more than 2,048
cells), each softened by its own R_max, summed at every cell's centre:
|a_c| = |sum_k M_k (Z_k - Z_c) / (|Z_k - Z_c|^2 + R_k^2)^(3/2)|, the term of a
source at zero softened distance dropped.
"""
from __future__ import annotations

import numpy as np

from . import mlp

ABSOLUTE, RELATIVE = 0, 1


def _criterion(d2: float, ra: float, rb: float, theta: float) -> bool:
    th2 = theta * theta
    s = ra + rb
    return th2 * d2 >= s * s


def cell_parts(o):
    """Per-cell feature parts from the oracle's geometry: (log10 R_max,
    log10 M, log10 trace-free quadrupole norm term, body count)."""
    M, Z, R, mom = o.geometry()
    cnt = o.cells().count.astype(np.float64)
    # moments in multi-index order: M, dipole (3), then Qxx Qxy Qxz Qyy Qyz Qzz
    Q = mom[:, 4:10]
    tr = (Q[:, 0] + Q[:, 3] + Q[:, 5]) / 3.0
    n2 = ((Q[:, 0] - tr) ** 2 + (Q[:, 3] - tr) ** 2 + (Q[:, 5] - tr) ** 2
          + 2.0 * (Q[:, 1] ** 2 + Q[:, 2] ** 2 + Q[:, 4] ** 2))
    den = M * R * R
    ok = (den > 0) & (cnt > 1)  # a cell of one body has no quadrupole
    with np.errstate(divide="ignore", invalid="ignore"):
        qn = np.where(ok, np.sqrt(n2) / np.where(ok, den, 1.0), 0.0)
        lgR = np.log10(R)
    return lgR, np.log10(M), np.log10(qn + 1e-12), cnt


def field_estimate(o):
    """log10 |a_c| at every cell from the softened monopoles of the coarse
    level (definition in the module docstring)."""
    M, Z, R, _ = o.geometry()
    lev = o.cells().level
    depth = int(lev.max())
    L = 0
    for l in range(depth + 1):
        if int((lev == l).sum()) > 2048:
            break
        L = l
    src = np.nonzero(lev == L)[0]
    a = np.zeros((Z.shape[0], 3))
    for k in src:
        d = Z[k][None, :] - Z
        r2 = (d * d).sum(1) + R[k] * R[k]
        w = np.zeros_like(r2)
        nz = r2 > 0
        w[nz] = M[k] / (r2[nz] * np.sqrt(r2[nz]))
        a += w[:, None] * d
    return np.log10(np.linalg.norm(a, axis=1) + 1e-30)


def pair_features(o, pairs, parts=None):
    """Raw features [K, 8] of cell pairs [K, 2], and the pairs as ordered for
    the features (K x 2)."""
    lgR, lgM, lgq, cnt = parts if parts is not None else cell_parts(o)
    _, Z, R, _ = o.geometry()
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    A, B = pairs[:, 0].copy(), pairs[:, 1].copy()
    ra, rb = R[A].astype(np.float32), R[B].astype(np.float32)
    swap = (rb > ra) | ((rb == ra) & (B < A))
    A[swap], B[swap] = pairs[swap, 1], pairs[swap, 0]
    d = Z[A] - Z[B]
    lr = 0.5 * np.log10((d * d).sum(1))
    f = np.empty((pairs.shape[0], 8))
    f[:, 0] = lr
    f[:, 1] = np.maximum(lgR[A] - lr, -12.0)
    f[:, 2] = np.maximum(lgR[B] - lr, -12.0)
    f[:, 3] = lgM[A]
    f[:, 4] = lgM[B]
    f[:, 5] = lgq[A]
    f[:, 6] = lgq[B]
    f[:, 7] = np.log10(cnt[A] + cnt[B])
    return f, np.stack([A, B], 1)


def walk(o, params, log10_target: float, theta_max: float = 1.0, min_work: int = 256, rule: int = RELATIVE,
         decide=None):
    """The selector walk over the oracle's tree at the oracle's theta.

    ``decide(A, B, score)`` (optional) overrides the decision of a scored
    pair; by default the pair is accepted when score < log10_target.
    Returns (m2l[K,2], p2p[K,2], self[K]) with pairs as (min, max), and a
    dict of every scored pair -> score."""
    cells = o.cells()
    nchild, first = cells.nchild, cells.first_child
    count, level = cells.count.astype(np.int64), cells.level
    _, Z, R, _ = o.geometry()
    theta = o.theta
    parts = cell_parts(o)
    lga = field_estimate(o) if rule == RELATIVE else None
    lgM = parts[1]
    m2l, p2p, slf = [], [], []
    scores = {}
    front = [(0, 0)]
    while front:
        nxt = []
        # scores of the band pairs of this generation, in one network call
        band = []
        sep = {}
        for A, B in front:
            if A == B:
                continue
            d = Z[A] - Z[B]
            d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
            s_lo = _criterion(d2, R[A], R[B], theta)
            sep[(A, B)] = s_lo
            if (not s_lo and count[A] * count[B] >= min_work
                    and _criterion(d2, R[A], R[B], theta_max)):
                band.append((A, B))
        sc = {}
        if band:
            f, ordered = pair_features(o, band, parts)
            pred, _, _ = mlp.forward(params, f.astype(np.float32), "bf16")
            pred = np.asarray(pred, dtype=np.float64)
            l2r = 2.0 * f[:, 0]
            a_, b_ = ordered[:, 0], ordered[:, 1]
            if rule == RELATIVE:
                adj = np.maximum(lgM[b_] - l2r - lga[a_], lgM[a_] - l2r - lga[b_])
            else:
                adj = np.maximum(lgM[b_], lgM[a_]) - l2r
            for k, pr in enumerate(band):
                sc[pr] = float(pred[k] + adj[k])
                scores[(min(pr), max(pr))] = sc[pr]
        for A, B in front:
            if A == B:
                if nchild[A] == 0:
                    slf.append(A)
                    continue
                f0, k = int(first[A]), int(nchild[A])
                for i in range(k):
                    nxt.append((f0 + i, f0 + i))
                for i in range(k):
                    for j in range(i + 1, k):
                        nxt.append((f0 + i, f0 + j))
                continue
            acc = sep[(A, B)]
            if not acc and (A, B) in sc:
                s = sc[(A, B)]
                acc = bool(decide(A, B, s)) if decide is not None else s < log10_target
            if acc:
                m2l.append((min(A, B), max(A, B)))
                continue
            la, lb = nchild[A] == 0, nchild[B] == 0
            if la and lb:
                p2p.append((min(A, B), max(A, B)))
                continue
            if la:
                split, other = B, A
            elif lb:
                split, other = A, B
            else:
                if R[A] != R[B]:
                    pick_a = R[A] > R[B]
                elif level[A] != level[B]:
                    pick_a = level[A] < level[B]
                else:
                    pick_a = A < B
                split, other = (A, B) if pick_a else (B, A)
            for c in range(int(first[split]), int(first[split]) + int(nchild[split])):
                nxt.append((c, other))
        front = nxt
    return (np.array(m2l, dtype=np.int32).reshape(-1, 2), np.array(p2p, dtype=np.int32).reshape(-1, 2),
            np.array(slf, dtype=np.int32), scores)


def canonical(m2l, p2p, slf):
    """Lists sorted for comparison (pairs as (min, max), lexicographic)."""
    def srt(a):
        a = np.sort(np.asarray(a, dtype=np.int64).reshape(-1, 2), axis=1)
        return a[np.lexsort((a[:, 1], a[:, 0]))] if a.size else a
    return srt(m2l), srt(p2p), np.sort(np.asarray(slf, dtype=np.int64))
