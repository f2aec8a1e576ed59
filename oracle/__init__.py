"""FP64 CPU oracle of the angular-momentum-conserving Cartesian FMM.

TEST INFRASTRUCTURE ONLY: the product library never imports this package.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may load it.  It shares no code with the CUDA path.

The numerical work lives in ``fmm_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module compiles it on first use and wraps it with
ctypes + numpy.  What each routine follows is listed in the C file's header:
Sec. 2 (tree, opening criterion, Eqs. 1-4, 7, 8), App. A (general order) and
Sec. 3 (direct summation, balance metric, relative errors).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_HDR = os.path.join(_HERE, "fmm_oracle.h")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

UC, TC, TCO = 0, 1, 2
PART_FAR, PART_NEAR = 1, 2
VARIANTS = {"UC": UC, "TC": TC, "TCO": TCO}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liborc.so`` (gcc, -O2, no FP contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [I, P, P, P, P, I, D, I, P]
            lib.orc_destroy.argtypes = [P]
            for name in ("orc_sizes", "orc_get_keys", "orc_get_cells", "orc_get_geometry",
                         "orc_get_lists", "orc_eval", "orc_pair_accel", "orc_morton",
                         "orc_dtensor_generic", "orc_dtensor_p3", "orc_direct", "orc_balance",
                         "orc_set_lists", "orc_set_softening"):
                getattr(lib, name).restype = I
            lib.orc_sizes.argtypes = [P, P]
            lib.orc_get_keys.argtypes = [P, P, P, P, P]
            lib.orc_get_cells.argtypes = [P, P, P, P, P, P, P]
            lib.orc_get_geometry.argtypes = [P, P, P, P, P]
            lib.orc_get_lists.argtypes = [P, P, P, P]
            lib.orc_set_lists.argtypes = [P, P, I, P, I, P, I]
            lib.orc_eval.argtypes = [P, I, I, I, P, P, P, P]
            lib.orc_pair_accel.argtypes = [P, I, I, I, I, P, P, P]
            lib.orc_morton.argtypes = [I, P, P, P, P, P, P]
            lib.orc_dtensor_generic.argtypes = [P, D, I, P]
            lib.orc_dtensor_p3.argtypes = [P, D, P, P, P, P, P, P]
            lib.orc_direct.argtypes = [I, P, P, P, P, I, P, D, P, P, P]
            lib.orc_set_softening.argtypes = [P, D]
            lib.orc_balance.argtypes = [I, P, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


@dataclass
class Cells:
    begin: np.ndarray
    count: np.ndarray
    level: np.ndarray
    parent: np.ndarray
    first_child: np.ndarray
    nchild: np.ndarray


class Oracle:
    """One tree (Sec. 2) over caller-order bodies, with its interaction lists.

    ``Oracle(x, y, z, m, theta, n_crit=25, P=3)`` sorts, builds the octree,
    computes Z, R_max and the moments to order P, and walks the tree.
    """

    def __init__(self, x, y, z, m, theta: float, n_crit: int = 25, P: int = 3, softening: float = 0.0):
        lib = _load()
        self.x, self.y, self.z, self.m = (_f64(a) for a in (x, y, z, m))
        self.n = int(self.x.shape[0])
        self.theta, self.n_crit, self.P = float(theta), int(n_crit), int(P)
        err = ctypes.c_int(0)
        h = lib.orc_create(self.n, _ptr(self.x), _ptr(self.y), _ptr(self.z), _ptr(self.m),
                           self.n_crit, self.theta, self.P, ctypes.byref(err))
        if not h:
            raise OracleError(f"orc_create failed ({err.value})")
        self._h = ctypes.c_void_p(h)
        sz = np.zeros(6, dtype=np.int32)
        lib.orc_sizes(self._h, _ptr(sz))
        (_, self.ncell, self.n_m2l, self.n_p2p, self.n_self, self.nmom) = (int(v) for v in sz)
        self.softening = 0.0
        if softening:
            self.set_softening(softening)

    def set_softening(self, eps: float):
        """Plummer softening of the forces (G = -1/sqrt(R^2 + eps^2)); the
        tree and the lists do not depend on it."""
        if _load().orc_set_softening(self._h, float(eps)) != 0:
            raise OracleError("softening must be finite and >= 0")
        self.softening = float(eps)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    # ---- intermediate results -------------------------------------------
    def keys(self):
        """(sorted keys u64, order i32 sorted->caller, lo[3], scale)."""
        key = np.zeros(self.n, dtype=np.uint64)
        order = np.zeros(self.n, dtype=np.int32)
        lo = np.zeros(3)
        scale = np.zeros(1)
        _load().orc_get_keys(self._h, _ptr(key), _ptr(order), _ptr(lo), _ptr(scale))
        return key, order, lo, float(scale[0])

    def cells(self) -> Cells:
        arrs = [np.zeros(self.ncell, dtype=np.int32) for _ in range(6)]
        _load().orc_get_cells(self._h, *(_ptr(a) for a in arrs))
        return Cells(*arrs)

    def geometry(self):
        """(M[ncell], Z[ncell,3], Rmax[ncell], moments[ncell, nmom])."""
        M = np.zeros(self.ncell)
        Z = np.zeros((self.ncell, 3))
        R = np.zeros(self.ncell)
        mom = np.zeros((self.ncell, self.nmom))
        _load().orc_get_geometry(self._h, _ptr(M), _ptr(Z), _ptr(R), _ptr(mom))
        return M, Z, R, mom

    def lists(self):
        """(m2l[K,2], p2p[K,2], self[K]) in walk order, each pair (min, max)."""
        m2l = np.zeros((self.n_m2l, 2), dtype=np.int32)
        p2p = np.zeros((self.n_p2p, 2), dtype=np.int32)
        slf = np.zeros(self.n_self, dtype=np.int32)
        _load().orc_get_lists(self._h, _ptr(m2l), _ptr(p2p), _ptr(slf))
        return m2l, p2p, slf

    def set_lists(self, m2l, p2p, slf):
        """Replaces the interaction lists (another pair selection over the same
        tree); ``accel`` then sums those pairs."""
        m2l = np.ascontiguousarray(np.asarray(m2l, dtype=np.int32).reshape(-1, 2))
        p2p = np.ascontiguousarray(np.asarray(p2p, dtype=np.int32).reshape(-1, 2))
        slf = np.ascontiguousarray(np.asarray(slf, dtype=np.int32).reshape(-1))
        rc = _load().orc_set_lists(self._h, _ptr(m2l), m2l.shape[0], _ptr(p2p), p2p.shape[0], _ptr(slf),
                                   slf.shape[0])
        if rc != 0:
            raise OracleError(f"orc_set_lists failed ({rc})")
        self.n_m2l, self.n_p2p, self.n_self = m2l.shape[0], p2p.shape[0], slf.shape[0]

    # ---- forces ----------------------------------------------------------
    def accel(self, variant="TC", generic=False, parts=PART_FAR | PART_NEAR, targets=None) -> np.ndarray:
        """Accelerations [n,3] in caller order (G = 1).  With ``targets`` (caller
        indices) only those bodies are evaluated and the result is [len(targets), 3]."""
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        a = [np.zeros(self.n) for _ in range(3)]
        mask = None
        if targets is not None:
            targets = np.asarray(targets, dtype=np.int64)
            mask = np.zeros(self.n, dtype=np.uint8)
            mask[targets] = 1
        rc = _load().orc_eval(self._h, v, int(bool(generic)), int(parts),
                              _ptr(mask) if mask is not None else None, *(_ptr(c) for c in a))
        if rc != 0:
            raise OracleError(f"orc_eval failed ({rc})")
        out = np.stack(a, axis=1)
        return out if targets is None else out[targets]

    def pair_accel(self, A: int, B: int, variant="TC", generic=False) -> np.ndarray:
        v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        a = [np.zeros(self.n) for _ in range(3)]
        rc = _load().orc_pair_accel(self._h, int(A), int(B), v, int(bool(generic)),
                                    *(_ptr(c) for c in a))
        if rc != 0:
            raise OracleError(f"orc_pair_accel failed ({rc})")
        return np.stack(a, axis=1)

    def cell_bodies(self, c: int) -> np.ndarray:
        """Caller indices of the bodies of cell c."""
        if not hasattr(self, "_order"):
            self._order = self.keys()[1]
            self._cells = self.cells()
        b, n = int(self._cells.begin[c]), int(self._cells.count[c])
        return self._order[b:b + n]


# ---- free functions ---------------------------------------------------------
def morton(x, y, z):
    """Keys in caller order, cube origin lo[3] and scale (2^21 / extent)."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.shape[0]
    keys = np.zeros(n, dtype=np.uint64)
    lo = np.zeros(3)
    scale = np.zeros(1)
    rc = _load().orc_morton(n, _ptr(x), _ptr(y), _ptr(z), _ptr(keys), _ptr(lo), _ptr(scale))
    if rc != 0:
        raise OracleError(f"orc_morton failed ({rc})")
    return keys, lo, float(scale[0])


def dtensor_generic(r, n: int, eps: float = 0.0) -> np.ndarray:
    """Symmetric components of the n-th derivative of -1/sqrt(R^2 + eps^2),
    multi-index order."""
    r = _f64(r)
    out = np.zeros((n + 1) * (n + 2) // 2)
    _load().orc_dtensor_generic(_ptr(r), float(eps), int(n), _ptr(out))
    return out


def dtensor_p3(r, eps: float = 0.0):
    """(D, D_i, D_ij, D_ijk, D_ijkl, D'_ijkl) of -1/sqrt(R^2 + eps^2) as full arrays."""
    r = _f64(r)
    d0 = np.zeros(1)
    d1, d2, d3 = np.zeros(3), np.zeros((3, 3)), np.zeros((3, 3, 3))
    d4, d4p = np.zeros((3, 3, 3, 3)), np.zeros((3, 3, 3, 3))
    _load().orc_dtensor_p3(_ptr(r), float(eps), _ptr(d0), _ptr(d1), _ptr(d2), _ptr(d3), _ptr(d4), _ptr(d4p))
    return float(d0[0]), d1, d2, d3, d4, d4p


def multi_indices(n: int):
    """Exponent triples (a,b,c) of order n in the oracle's storage order."""
    return [(a, b, n - a - b) for a in range(n, -1, -1) for b in range(n - a, -1, -1)]


def direct(x, y, z, m, targets=None, eps: float = 0.0) -> np.ndarray:
    """Exact accelerations by Neumaier-compensated direct summation [nt,3]
    (softened by eps when eps > 0)."""
    x, y, z, m = (_f64(a) for a in (x, y, z, m))
    n = x.shape[0]
    t = np.arange(n, dtype=np.int32) if targets is None else np.ascontiguousarray(targets, dtype=np.int32)
    a = [np.zeros(t.shape[0]) for _ in range(3)]
    rc = _load().orc_direct(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), int(t.shape[0]), _ptr(t), float(eps),
                            *(_ptr(c) for c in a))
    if rc != 0:
        raise OracleError("orc_direct failed")
    return np.stack(a, axis=1)


def balance(x, y, z, m, acc) -> tuple[float, float]:
    """(net force balance, net torque balance) of Sec. 3."""
    x, y, z, m = (_f64(a) for a in (x, y, z, m))
    acc = np.asarray(acc, dtype=np.float64)
    ax, ay, az = (np.ascontiguousarray(acc[:, d]) for d in range(3))
    out = np.zeros(2)
    _load().orc_balance(x.shape[0], _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(ax), _ptr(ay),
                        _ptr(az), _ptr(out))
    return float(out[0]), float(out[1])


def force_errors(acc, ref) -> dict:
    """Relative force error eps_n = |g - g_PP| / |g_PP| (Sec. 3): mean and rms."""
    acc = np.asarray(acc, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    e = np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return {"mean": float(e.mean()), "rms": float(np.sqrt((e * e).mean())), "max": float(e.max())}


def torque_errors(pos, acc, ref) -> dict:
    """Relative torque error with X x g about the coordinate origin (Sec. 3)."""
    pos = np.asarray(pos, dtype=np.float64)
    t = np.cross(pos, acc)
    t0 = np.cross(pos, ref)
    e = np.linalg.norm(t - t0, axis=1) / np.linalg.norm(t0, axis=1)
    return {"mean": float(e.mean()), "rms": float(np.sqrt((e * e).mean()))}
