"""Thin ctypes binding of libamfmm.so (the C ABI of include/amfmm.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current CUDA stream.  The
binding raises if the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamfmm.so")

FMM_OK, FMM_EINVAL, FMM_ENOMEM, FMM_ECUDA, FMM_ETIMEOUT, FMM_EORDER, FMM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
UC, TC, TCO = 0, 1, 2
FP64, MIXED = 0, 1
VARIANTS = {"UC": UC, "TC": TC, "TCO": TCO}
PRECISIONS = {"fp64": FP64, "mixed": MIXED}
MOMENT_NAMES = ["M", "x", "y", "z", "xx", "xy", "xz", "yy", "yz", "zz", "xxx", "xxy", "xxz", "xyy",
                "xyz", "xzz", "yyy", "yyz", "yzz", "zzz"]

_lock = threading.Lock()
_lib = None


SELECTOR_RULES = {"absolute": 0, "relative": 1}


class FMMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("n_crit", ctypes.c_int), ("order_P", ctypes.c_int),
                ("variant", ctypes.c_int), ("precision", ctypes.c_int), ("G", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncell", ctypes.c_int64), ("nleaf", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("n_m2l", ctypes.c_int64), ("n_p2p", ctypes.c_int64),
                ("n_self", ctypes.c_int64), ("p2p_body_pairs", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("lo", ctypes.c_double * 3), ("scale", ctypes.c_double),
                ("ms_tree", ctypes.c_float), ("ms_upward", ctypes.c_float), ("ms_walk", ctypes.c_float),
                ("ms_m2l", ctypes.c_float), ("ms_p2p", ctypes.c_float), ("ms_reduce", ctypes.c_float),
                ("ms_downward", ctypes.c_float), ("n_scored", ctypes.c_int64)]


def load() -> ctypes.CDLL:
    """Loads libamfmm.so from the package directory (raises if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(LIB_PATH)
            P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            sig = {
                "fmm_create": [ctypes.POINTER(P), ctypes.POINTER(_Opts), P],
                "fmm_set_opts": [P, ctypes.POINTER(_Opts)],
                "fmm_set_timing": [P, I],
                "fmm_set_softening": [P, D],
                "fmm_set_tile": [P, I],
                "fmm_set_graph": [P, I],
                "fmm_graph_stats": [P, P],
                "fmm_autotune": [P, P, P, P, P, P, I, P, I, P, I, I, P, P, P, P, P, P],
                "fmm_build_tree": [P, P, P, P, P, I64, D],
                "fmm_upward": [P],
                "fmm_interact": [P],
                "fmm_downward": [P],
                "fmm_forces": [P, P, P, P],
                "fmm_solve": [P, P, P, P, P, I64, P, P, P],
                "fmm_solve_host": [P, P, P, P, P, I64, P, P, P],
                "fmm_get_stats": [P, ctypes.POINTER(_Stats)],
                "fmm_export_keys": [P, P, P],
                "fmm_export_tree": [P, P, P, P, P, P, P, P, P, P],
                "fmm_export_moments": [P, P],
                "fmm_export_lists": [P, P, P, P],
                "fmm_export_locals": [P, P],
                "fmm_direct": [P, P, P, P, P, I64, P, I64, P, P, P],
                "fmm_balance": [P, P, P, P, P, P, P, P, I64, P],
                "fmm_leapfrog": [P, P, P, P, P, P, P, P, I64, D, I, P, P, P, P],
                "fmm_solve_batch": [P, P, P, P, P, P, I, P, P, P],
                "fmm_autotune_ncrit": [P, P, P, P, P, P, I, P, I, I, P, P, P, P, P],
                "fmm_selector_set": [P, P, D, D, I64, I, I],
                "fmm_debug_walk_wait_timeout": [P],
                "fmm_selector_samples": [P, P, I64, P, P],
                "fmm_mlp_forward": [P, P, P, I64, P],
                "fmm_mlp_grad": [P, P, P, P, I64, P, P],
                "fmm_mlp_adam": [P, P, P, P, P, ctypes.c_float, I],
                "fmm_selector_train": [P, P, P, P, P, I64, I, I, ctypes.c_float, ctypes.c_ulonglong, P],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = I
            lib.fmm_alu_peak.argtypes = [I, I, ctypes.POINTER(ctypes.c_double)]
            lib.fmm_alu_peak.restype = I
            lib.fmm_selector_nparams.argtypes = []
            lib.fmm_selector_nparams.restype = I
            lib.fmm_graph_error.argtypes = [P]
            lib.fmm_graph_error.restype = ctypes.c_char_p
            lib.fmm_destroy.argtypes = [P]
            lib.fmm_destroy.restype = None
            lib.fmm_last_error.argtypes = [P]
            lib.fmm_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _dptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Stats:
    n: int
    ncell: int
    nleaf: int
    depth: int
    n_m2l: int
    n_p2p: int
    n_self: int
    p2p_body_pairs: int
    launches: int
    lo: tuple
    scale: float
    ms: dict
    n_scored: int = 0


def alu_peak(precision: str = "fp64", reps: int = 5) -> float:
    """Measured TFLOP/s of the plain FMA pipe (FP64 or FP32) on the current
    device (fmm_alu_peak)."""
    out = ctypes.c_double(0.0)
    rc = load().fmm_alu_peak(PRECISIONS[precision], int(reps), ctypes.byref(out))
    if rc != FMM_OK:
        raise FMMError(rc, "fmm_alu_peak failed")
    return float(out.value)


class FMM:
    """One solver context on the current CUDA device and stream.

    ``FMM(theta=0.5, n_crit=25, variant="TC", precision="fp64", G=1.0)``;
    ``solve(x, y, z, m)`` takes float64 CUDA tensors (caller order) and returns
    the accelerations (ax, ay, az).  The five stage methods mirror the C ABI.
    """

    def __init__(self, theta: float = 0.5, n_crit: int = 25, variant="TC", precision="fp64",
                 G: float = 1.0, order_P: int = 3, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.opts = _Opts(float(theta), int(n_crit), int(order_P),
                          VARIANTS[variant] if isinstance(variant, str) else int(variant),
                          PRECISIONS[precision] if isinstance(precision, str) else int(precision), float(G))
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = ctypes.c_void_p()
        rc = self.lib.fmm_create(ctypes.byref(h), ctypes.byref(self.opts), ctypes.c_void_p(s.cuda_stream))
        if rc != FMM_OK:
            raise FMMError(rc, "fmm_create failed")
        self._h = h
        self._bodies = None

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc != FMM_OK:
            msg = self.lib.fmm_last_error(self._h)
            raise FMMError(rc, f"{what}: {msg.decode() if msg else ''}")

    def set_opts(self, theta=None, n_crit=None, variant=None, precision=None, G=None):
        o = self.opts
        if theta is not None:
            o.theta = float(theta)
        if n_crit is not None:
            o.n_crit = int(n_crit)
        if variant is not None:
            o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        if precision is not None:
            o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if G is not None:
            o.G = float(G)
        self._check(self.lib.fmm_set_opts(self._h, ctypes.byref(o)), "fmm_set_opts")

    def set_softening(self, eps: float):
        """Plummer softening G = -1/sqrt(R^2 + eps^2) of the following solves
        and of direct(); 0 restores the unsoftened method."""
        self._check(self.lib.fmm_set_softening(self._h, float(eps)), "fmm_set_softening")

    def set_tile(self, rows: int):
        """Rows of a leaf staged per pass of the near field (8, 16 or 32)."""
        self._check(self.lib.fmm_set_tile(self._h, int(rows)), "fmm_set_tile")

    def set_timing(self, on: bool = True):
        self._check(self.lib.fmm_set_timing(self._h, int(bool(on))), "fmm_set_timing")

    def set_graph(self, on: bool = True):
        """Solves as one CUDA-graph launch (captured on the first solve of a
        configuration, replayed while the sizes stay the same)."""
        self._check(self.lib.fmm_set_graph(self._h, int(bool(on))), "fmm_set_graph")

    def graph_stats(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        self._check(self.lib.fmm_graph_stats(self._h, ctypes.cast(out, ctypes.c_void_p)), "fmm_graph_stats")
        return dict(replays=out[0], captures=out[1], fallbacks=out[2], capture_failures=out[3], kernels=out[4],
                    error=self.lib.fmm_graph_error(self._h).decode())

    # ---- stages ------------------------------------------------------------
    def _as_dev(self, a):
        t = self._torch
        a = a if isinstance(a, t.Tensor) else t.as_tensor(a)
        if a.dtype != t.float64 or not a.is_cuda or not a.is_contiguous():
            raise ValueError("body arrays must be contiguous float64 CUDA tensors")
        return a

    def build_tree(self, x, y, z, m, theta: float = 0.0):
        x, y, z, m = (self._as_dev(a) for a in (x, y, z, m))
        n = x.shape[0]
        if not (y.shape[0] == z.shape[0] == m.shape[0] == n):
            raise ValueError("x, y, z, m must have the same length")
        self._bodies = (x, y, z, m)  # read again by the later stages
        self._check(self.lib.fmm_build_tree(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), n,
                                            float(theta)), "fmm_build_tree")

    def upward(self):
        self._check(self.lib.fmm_upward(self._h), "fmm_upward")

    def interact(self):
        self._check(self.lib.fmm_interact(self._h), "fmm_interact")

    def downward(self):
        self._check(self.lib.fmm_downward(self._h), "fmm_downward")

    def forces(self, out=None):
        t = self._torch
        n = self._bodies[0].shape[0]
        if out is None:
            out = tuple(t.empty(n, dtype=t.float64, device=self._bodies[0].device) for _ in range(3))
        self._check(self.lib.fmm_forces(self._h, *(_dptr(o) for o in out)), "fmm_forces")
        return out

    def solve(self, x, y, z, m, out=None):
        x, y, z, m = (self._as_dev(a) for a in (x, y, z, m))
        t = self._torch
        n = x.shape[0]
        if out is None:
            out = tuple(t.empty(n, dtype=t.float64, device=x.device) for _ in range(3))
        self._bodies = (x, y, z, m)
        self._check(self.lib.fmm_solve(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), n,
                                       *(_dptr(o) for o in out)), "fmm_solve")
        return out

    def solve_host(self, x, y, z, m, out=None):
        """Solve from host arrays (numpy float64 or pinned CPU tensors)."""
        import numpy as np

        def hp(a):
            if isinstance(a, np.ndarray):
                if a.dtype != np.float64 or not a.flags.c_contiguous:
                    raise ValueError("host arrays must be contiguous float64")
                return ctypes.c_void_p(a.ctypes.data)
            return ctypes.c_void_p(a.data_ptr())

        n = x.shape[0]
        if out is None:
            out = tuple(np.empty(n) for _ in range(3))
        self._check(self.lib.fmm_solve_host(self._h, hp(x), hp(y), hp(z), hp(m), n, *(hp(o) for o in out)),
                    "fmm_solve_host")
        return out

    # ---- ensembles (a13) -------------------------------------------------------
    @staticmethod
    def _offsets(offsets):
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        return off, ctypes.c_void_p(off.ctypes.data)

    def solve_batch(self, x, y, z, m, offsets, out=None):
        """Independent systems in one launch sequence: system s owns bodies
        [offsets[s], offsets[s+1]) of the concatenated arrays."""
        t = self._torch
        x, y, z, m = (self._as_dev(a) for a in (x, y, z, m))
        off, offp = self._offsets(offsets)
        n = x.shape[0]
        if int(off[-1]) != n:
            raise ValueError("offsets[-1] must equal the number of bodies")
        if out is None:
            out = tuple(t.empty(n, dtype=t.float64, device=x.device) for _ in range(3))
        self._bodies = (x, y, z, m)
        self._check(self.lib.fmm_solve_batch(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), offp,
                                             len(off) - 1, *(_dptr(o) for o in out)), "fmm_solve_batch")
        return out

    def autotune_ncrit(self, x, y, z, m, offsets, candidates=(16, 25, 32, 64), reps: int = 3):
        """Times the batched solve for each leaf size; returns (best, {n_crit: ms})."""
        import numpy as np
        t = self._torch
        x, y, z, m = (self._as_dev(a) for a in (x, y, z, m))
        off, offp = self._offsets(offsets)
        cand = np.ascontiguousarray(candidates, dtype=np.int32)
        ms = np.zeros(len(cand), dtype=np.float32)
        best = ctypes.c_int(0)
        out = tuple(t.empty(x.shape[0], dtype=t.float64, device=x.device) for _ in range(3))
        self._bodies = (x, y, z, m)
        self._check(self.lib.fmm_autotune_ncrit(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), offp, len(off) - 1,
                                                ctypes.c_void_p(cand.ctypes.data), len(cand), int(reps),
                                                *(_dptr(o) for o in out), ctypes.byref(best),
                                                ctypes.c_void_p(ms.ctypes.data)), "fmm_autotune_ncrit")
        return int(best.value), {int(k): float(v) for k, v in zip(cand, ms)}

    def autotune(self, x, y, z, m, offsets, ncrit=(16, 25, 32, 64), tiles=(8, 16, 32), reps: int = 3):
        """Times the batched solve for every (n_crit, tile) pair; returns
        (best n_crit, best tile, {(n_crit, tile): ms})."""
        import numpy as np
        t = self._torch
        x, y, z, m = (self._as_dev(a) for a in (x, y, z, m))
        off, offp = self._offsets(offsets)
        nc = np.ascontiguousarray(ncrit, dtype=np.int32)
        tl = np.ascontiguousarray(tiles, dtype=np.int32)
        ms = np.zeros(len(nc) * len(tl), dtype=np.float32)
        bn, bt = ctypes.c_int(0), ctypes.c_int(0)
        out = tuple(t.empty(x.shape[0], dtype=t.float64, device=x.device) for _ in range(3))
        self._bodies = (x, y, z, m)
        self._check(self.lib.fmm_autotune(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), offp, len(off) - 1,
                                          ctypes.c_void_p(nc.ctypes.data), len(nc), ctypes.c_void_p(tl.ctypes.data),
                                          len(tl), int(reps), *(_dptr(o) for o in out), ctypes.byref(bn),
                                          ctypes.byref(bt), ctypes.c_void_p(ms.ctypes.data)), "fmm_autotune")
        table = {(int(a), int(b)): float(ms[i * len(tl) + j]) for i, a in enumerate(nc) for j, b in enumerate(tl)}
        return int(bn.value), int(bt.value), table

    # ---- learned pair selector (a12) -------------------------------------------
    def selector_nparams(self) -> int:
        return int(self.lib.fmm_selector_nparams())

    def selector_set(self, params, log10_target: float, enable: bool = True, theta_max: float = 1.0,
                     min_work: int = 256, rule: str = "relative"):
        """Learned selection in the band (theta, theta_max] for pairs with
        n_A n_B >= min_work: accepted when the predicted pair error (absolute,
        or relative to the field at each side) is below 10**log10_target."""
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32) if params is not None else None
        if enable and (p is None or p.shape[0] != self.selector_nparams()):
            raise ValueError("params must hold fmm_selector_nparams() floats")
        self._check(self.lib.fmm_selector_set(self._h, ctypes.c_void_p(p.ctypes.data) if p is not None else None,
                                              float(log10_target), float(theta_max), int(min_work),
                                              SELECTOR_RULES[rule], int(bool(enable))),
                    "fmm_selector_set")

    def selector_samples(self, pairs, labels: bool = True):
        """Raw features [K, 8] (and labels [K]) of cell pairs of the current tree."""
        t = self._torch
        pr = t.as_tensor(pairs, dtype=t.int32, device=self._bodies[0].device).contiguous()
        K = pr.shape[0]
        feat = t.empty((K, 8), dtype=t.float32, device=pr.device)
        lab = t.empty(K, dtype=t.float32, device=pr.device) if labels else None
        self._check(self.lib.fmm_selector_samples(self._h, _dptr(pr), K, _dptr(feat), _dptr(lab) if labels else None),
                    "fmm_selector_samples")
        return feat, lab

    def mlp_forward(self, params, feat):
        t = self._torch
        out = t.empty(feat.shape[0], dtype=t.float32, device=feat.device)
        self._check(self.lib.fmm_mlp_forward(self._h, _dptr(params), _dptr(feat.contiguous()), feat.shape[0],
                                             _dptr(out)), "fmm_mlp_forward")
        return out

    def mlp_grad(self, params, feat, label):
        t = self._torch
        g = t.empty(params.shape[0], dtype=t.float32, device=feat.device)
        loss = t.empty(1, dtype=t.float32, device=feat.device)
        self._check(self.lib.fmm_mlp_grad(self._h, _dptr(params), _dptr(feat.contiguous()), _dptr(label.contiguous()),
                                          feat.shape[0], _dptr(g), _dptr(loss)), "fmm_mlp_grad")
        return g, loss

    def selector_train(self, params, X, y, batch: int, steps: int, lr: float, seed: int = 0, adam=None):
        """Adam on minibatches (params: device float32 tensor, updated in place)."""
        import numpy as np
        t = self._torch
        if adam is None:
            adam = t.zeros(2 * params.shape[0], dtype=t.float32, device=params.device)
        losses = np.zeros(max(steps, 1), dtype=np.float32)
        self._check(self.lib.fmm_selector_train(self._h, _dptr(params), _dptr(adam), _dptr(X.contiguous()),
                                                _dptr(y.contiguous()), X.shape[0], int(batch), int(steps),
                                                float(lr), int(seed), ctypes.c_void_p(losses.ctypes.data)),
                    "fmm_selector_train")
        return losses[:steps], adam

    # ---- time integration (a14) ---------------------------------------------
    def leapfrog(self, x, y, z, vx, vy, vz, m, dt: float, nsteps: int, acc=None, record=True):
        """Uniform kick-drift-kick steps, state updated in place.  Returns
        (ax, ay, az) and, if record, a [nsteps+1, 6] tensor of the totals
        (P_x, P_y, P_z, L_x, L_y, L_z) after every step."""
        t = self._torch
        arrs = [self._as_dev(a) for a in (x, y, z, vx, vy, vz, m)]
        n = arrs[0].shape[0]
        if acc is None:
            acc = tuple(t.empty(n, dtype=t.float64, device=arrs[0].device) for _ in range(3))
        mom = t.zeros((nsteps + 1, 6), dtype=t.float64, device=arrs[0].device) if record else None
        self._bodies = (arrs[0], arrs[1], arrs[2], arrs[6])
        self._check(self.lib.fmm_leapfrog(self._h, *(_dptr(a) for a in arrs), n, float(dt), int(nsteps),
                                          *(_dptr(a) for a in acc), _dptr(mom) if record else None),
                    "fmm_leapfrog")
        return acc, mom

    def debug_walk_wait_timeout(self) -> int:
        """Return code of fmm_debug_walk_wait_timeout (FMM_ETIMEOUT expected)."""
        return int(self.lib.fmm_debug_walk_wait_timeout(self._h))

    # ---- diagnostics (Sec. 3) ---------------------------------------------------
    def direct(self, x, y, z, m, targets):
        """Exact FP64 accelerations of the target bodies by direct summation."""
        t = self._torch
        x, y, z, m = (self._as_dev(a) for a in (x, y, z, m))
        tg = t.as_tensor(targets, dtype=t.int32, device=x.device).contiguous()
        out = tuple(t.empty(tg.shape[0], dtype=t.float64, device=x.device) for _ in range(3))
        self._check(self.lib.fmm_direct(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), x.shape[0],
                                        _dptr(tg), tg.shape[0], *(_dptr(o) for o in out)), "fmm_direct")
        return out

    def balance(self, x, y, z, m, ax, ay, az):
        """(net force balance, net torque balance) of Sec. 3."""
        x, y, z, m, ax, ay, az = (self._as_dev(a) for a in (x, y, z, m, ax, ay, az))
        out = (ctypes.c_double * 2)()
        self._check(self.lib.fmm_balance(self._h, _dptr(x), _dptr(y), _dptr(z), _dptr(m), _dptr(ax), _dptr(ay),
                                         _dptr(az), x.shape[0], ctypes.cast(out, ctypes.c_void_p)), "fmm_balance")
        return float(out[0]), float(out[1])

    # ---- introspection -------------------------------------------------------
    def stats(self) -> Stats:
        s = _Stats()
        self._check(self.lib.fmm_get_stats(self._h, ctypes.byref(s)), "fmm_get_stats")
        ms = {k: float(getattr(s, "ms_" + k)) for k in ("tree", "upward", "walk", "m2l", "p2p", "reduce",
                                                         "downward")}
        return Stats(s.n, s.ncell, s.nleaf, s.depth, s.n_m2l, s.n_p2p, s.n_self, s.p2p_body_pairs,
                     s.launches, tuple(s.lo), s.scale, ms, s.n_scored)

    def export_keys(self):
        t = self._torch
        n = self._bodies[0].shape[0]
        dev = self._bodies[0].device
        keys = t.empty(n, dtype=t.int64, device=dev)
        order = t.empty(n, dtype=t.int32, device=dev)
        self._check(self.lib.fmm_export_keys(self._h, _dptr(keys), _dptr(order)), "fmm_export_keys")
        return keys, order

    def export_tree(self, geometry: bool = True):
        t = self._torch
        st = self.stats()
        nc = st.ncell
        dev = self._bodies[0].device
        ints = [t.empty(nc, dtype=t.int32, device=dev) for _ in range(6)]
        if geometry:
            M = t.empty(nc, dtype=t.float64, device=dev)
            Z = t.empty((nc, 3), dtype=t.float64, device=dev)
            R = t.empty(nc, dtype=t.float64, device=dev)
            g = [_dptr(M), _dptr(Z), _dptr(R)]
        else:
            M = Z = R = None
            g = [None, None, None]
        self._check(self.lib.fmm_export_tree(self._h, *(_dptr(a) for a in ints), *g), "fmm_export_tree")
        names = ["begin", "count", "level", "parent", "first_child", "nchild"]
        out = dict(zip(names, ints))
        out.update(M=M, Z=Z, Rmax=R)
        return out

    def _mom_stride(self):
        P = self.opts.order_P
        return (P + 1) * (P + 2) * (P + 3) // 6

    def export_moments(self):
        t = self._torch
        nc = self.stats().ncell
        mom = t.empty((nc, self._mom_stride()), dtype=t.float64, device=self._bodies[0].device)
        self._check(self.lib.fmm_export_moments(self._h, _dptr(mom)), "fmm_export_moments")
        return mom

    def export_lists(self):
        t = self._torch
        st = self.stats()
        dev = self._bodies[0].device
        m2l = t.empty((max(st.n_m2l, 1), 2), dtype=t.int32, device=dev)
        p2p = t.empty((max(st.n_p2p, 1), 2), dtype=t.int32, device=dev)
        slf = t.empty(max(st.n_self, 1), dtype=t.int32, device=dev)
        self._check(self.lib.fmm_export_lists(self._h, _dptr(m2l), _dptr(p2p), _dptr(slf)), "fmm_export_lists")
        return m2l[:st.n_m2l], p2p[:st.n_p2p], slf[:st.n_self]

    def export_locals(self):
        t = self._torch
        nc = self.stats().ncell
        width = 20 if self.opts.order_P == 3 else self._mom_stride() - 1
        C = t.empty((nc, width), dtype=t.float64, device=self._bodies[0].device)
        self._check(self.lib.fmm_export_locals(self._h, _dptr(C)), "fmm_export_locals")
        return C
