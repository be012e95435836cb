"""FP64 CPU oracle for ADP-beta / MAID (arXiv 2502.09758) -- ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never imports it and shares no code with it.

Every function takes float64 NumPy arrays: images planar ``(C, H, W)``, kernels
``(C, K, K)``.  The C source (``oracle.c``) is compiled with gcc on first use
(or by ``build()``) into ``_liboracle.so`` next to this file.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")

REG_HUBER, REG_SQRT, REG_QUAD = 0, 1, 2


class _Prob(ct.Structure):
    _fields_ = [("C", ct.c_int), ("H", ct.c_int), ("W", ct.c_int), ("K", ct.c_int),
                ("alpha", ct.c_double), ("reg_param", ct.c_double), ("reg", ct.c_int),
                ("beta", ct.c_double), ("w0", ct.c_double)]


class MaidState(ct.Structure):
    """Mirror of ``orc_maid`` (Algorithm 2 state and the last call's report)."""
    _fields_ = [("eps", ct.c_double), ("delta", ct.c_double), ("step", ct.c_double),
                ("lam", ct.c_double), ("rho_up", ct.c_double), ("rho_down", ct.c_double),
                ("nu_up", ct.c_double), ("nu_down", ct.c_double), ("L_gx", ct.c_double),
                ("eps_stop", ct.c_double),
                ("max_bt", ct.c_int), ("max_rounds", ct.c_int), ("ll_max_iters", ct.c_int),
                ("cg_max_iters", ct.c_int), ("k", ct.c_int),
                ("accepted", ct.c_int), ("rounds", ct.c_int), ("trials", ct.c_int),
                ("ll_iters", ct.c_int), ("cg_iters", ct.c_int), ("ll_capped", ct.c_int),
                ("cg_capped", ct.c_int), ("stopped", ct.c_int),
                ("loss", ct.c_double), ("gradx_norm", ct.c_double), ("znorm", ct.c_double),
                ("psi", ct.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (plain -O2, IEEE semantics kept)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        d = ct.c_double
        P = ct.POINTER(_Prob)
        dp = ct.POINTER(ct.c_double)
        sig = {
            "orc_conv": (None, [P, dp, dp, dp]),
            "orc_conv_adj": (None, [P, dp, dp, dp]),
            "orc_dh": (None, [P, dp, dp]), "orc_dv": (None, [P, dp, dp]),
            "orc_dh_adj": (None, [P, dp, dp]), "orc_dv_adj": (None, [P, dp, dp]),
            "orc_phi": (d, [P, d]), "orc_dphi": (d, [P, d]), "orc_ddphi": (d, [P, d]),
            "orc_J": (d, [P, dp]), "orc_gradJ": (None, [P, dp, dp]),
            "orc_hessJ_vec": (None, [P, dp, dp, dp]),
            "orc_h": (d, [P, dp, dp, dp]), "orc_grad_h": (None, [P, dp, dp, dp, dp]),
            "orc_hess_h_vec": (None, [P, dp, dp, dp, dp]),
            "orc_lipschitz": (d, [P, dp, ct.c_int]),
            "orc_fista": (ct.c_int, [P, dp, dp, dp, d, ct.c_int, dp]),
            "orc_cg": (ct.c_int, [P, dp, dp, dp, d, ct.c_int, dp, dp, ct.POINTER(ct.c_int)]),
            "orc_cross_t": (None, [P, dp, dp, dp, dp, dp]),
            "orc_g": (d, [P, dp, dp, dp, dp]),
            "orc_r": (d, [P, dp, dp, dp]),
            "orc_upper": (d, [P, dp, dp, dp, dp, dp]),
            "orc_hypergrad": (ct.c_int, [P, dp, dp, dp, dp, dp, d, ct.c_int, dp, dp, dp,
                                         ct.POINTER(ct.c_int)]),
            "orc_maid_init": (None, [ct.POINTER(MaidState)]),
            "orc_maid_step": (ct.c_int, [P, ct.POINTER(MaidState), dp, dp, dp, dp, dp]),
            "orc_L_gx": (d, [P, dp]),
            "orc_norm": (d, [dp, ct.c_long]),
            "orc_conv_at": (d, [P, dp, dp, ct.c_int, ct.c_int, ct.c_int]),
            "orc_conv_adj_at": (d, [P, dp, dp, ct.c_int, ct.c_int, ct.c_int]),
            "orc_grad_h_at": (d, [P, dp, dp, dp, ct.c_int, ct.c_int, ct.c_int]),
            "orc_hess_h_vec_at": (d, [P, dp, dp, dp, ct.c_int, ct.c_int, ct.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle takes C-contiguous float64"
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Problem:
    """Shapes and weights of one ADP-beta instance (Eq. 2.5)."""
    C: int
    H: int
    W: int
    K: int
    alpha: float = 1e-2
    reg_param: float = 1e-2
    reg: int = REG_HUBER
    beta: float = 0.3
    w0: float = 1.0

    def _s(self):
        return ct.byref(_Prob(self.C, self.H, self.W, self.K, self.alpha, self.reg_param,
                              self.reg, self.beta, self.w0))

    @property
    def img_shape(self):
        return (self.C, self.H, self.W)

    @property
    def ker_shape(self):
        return (self.C, self.K, self.K)

    # ----------------------------------------------------------- operators
    def conv(self, b, x):
        b, x = _f64(b), _f64(x)
        out = np.empty(self.img_shape)
        _L().orc_conv(self._s(), _ptr(b), _ptr(x), _ptr(out))
        return out

    def conv_adj(self, b, z):
        b, z = _f64(b), _f64(z)
        out = np.empty(self.img_shape)
        _L().orc_conv_adj(self._s(), _ptr(b), _ptr(z), _ptr(out))
        return out

    # single outputs at sampled indices (rows of ``idx`` are (c, i, j))
    def conv_at(self, b, x, idx):
        b, x = _f64(b), _f64(x)
        return np.array([_L().orc_conv_at(self._s(), _ptr(b), _ptr(x), int(c), int(i), int(j))
                         for c, i, j in idx])

    def conv_adj_at(self, b, z, idx):
        b, z = _f64(b), _f64(z)
        return np.array([_L().orc_conv_adj_at(self._s(), _ptr(b), _ptr(z), int(c), int(i), int(j))
                         for c, i, j in idx])

    def grad_h_at(self, b, x, y, idx):
        b, x, y = _f64(b), _f64(x), _f64(y)
        return np.array([_L().orc_grad_h_at(self._s(), _ptr(b), _ptr(x), _ptr(y), int(c), int(i), int(j))
                         for c, i, j in idx])

    def hess_h_vec_at(self, b, x, v, idx):
        b, x, v = _f64(b), _f64(x), _f64(v)
        return np.array([_L().orc_hess_h_vec_at(self._s(), _ptr(b), _ptr(x), _ptr(v), int(c), int(i), int(j))
                         for c, i, j in idx])

    def _unary(self, name, x):
        x = _f64(x)
        out = np.empty(self.img_shape)
        getattr(_L(), name)(self._s(), _ptr(x), _ptr(out))
        return out

    def dh(self, x): return self._unary("orc_dh", x)
    def dv(self, x): return self._unary("orc_dv", x)
    def dh_adj(self, w): return self._unary("orc_dh_adj", w)
    def dv_adj(self, w): return self._unary("orc_dv_adj", w)

    def phi(self, t): return _L().orc_phi(self._s(), float(t))
    def dphi(self, t): return _L().orc_dphi(self._s(), float(t))
    def ddphi(self, t): return _L().orc_ddphi(self._s(), float(t))

    def J(self, x): return _L().orc_J(self._s(), _ptr(_f64(x)))
    def gradJ(self, x): return self._unary("orc_gradJ", x)

    def hessJ_vec(self, x, v):
        x, v = _f64(x), _f64(v)
        out = np.empty(self.img_shape)
        _L().orc_hessJ_vec(self._s(), _ptr(x), _ptr(v), _ptr(out))
        return out

    # --------------------------------------------------------- lower level
    def h(self, b, x, y):
        return _L().orc_h(self._s(), _ptr(_f64(b)), _ptr(_f64(x)), _ptr(_f64(y)))

    def grad_h(self, b, x, y):
        b, x, y = _f64(b), _f64(x), _f64(y)
        out = np.empty(self.img_shape)
        _L().orc_grad_h(self._s(), _ptr(b), _ptr(x), _ptr(y), _ptr(out))
        return out

    def hess_h_vec(self, b, x, v):
        b, x, v = _f64(b), _f64(x), _f64(v)
        out = np.empty(self.img_shape)
        _L().orc_hess_h_vec(self._s(), _ptr(b), _ptr(x), _ptr(v), _ptr(out))
        return out

    def lipschitz(self, b, c):
        return _L().orc_lipschitz(self._s(), _ptr(_f64(b)), int(c))

    def fista(self, b, y, x0, eps, max_iters=300):
        """Returns (x~, updates, ||grad_x h(x~)||)."""
        b, y = _f64(b), _f64(y)
        x = _f64(x0).copy()
        gn = ct.c_double()
        it = _L().orc_fista(self._s(), _ptr(b), _ptr(y), _ptr(x), float(eps), int(max_iters),
                            ct.byref(gn))
        return x, it, gn.value

    def cg(self, b, x, rhs, delta, max_iters=1000, q0=None):
        """Returns (q, iterations, residual norm, capped)."""
        b, x, rhs = _f64(b), _f64(x), _f64(rhs)
        q = np.zeros(self.img_shape) if q0 is None else _f64(q0).copy()
        res = ct.c_double()
        capped = ct.c_int()
        it = _L().orc_cg(self._s(), _ptr(b), _ptr(x), _ptr(rhs), float(delta), int(max_iters),
                         _ptr(q), ct.byref(res), ct.byref(capped))
        return q, it, res.value, bool(capped.value)

    def cross_t(self, b, x, y, q):
        b, x, y, q = _f64(b), _f64(x), _f64(y), _f64(q)
        out = np.empty(self.ker_shape)
        _L().orc_cross_t(self._s(), _ptr(b), _ptr(x), _ptr(y), _ptr(q), _ptr(out))
        return out

    # --------------------------------------------------------- upper level
    def g(self, a, x, y):
        """Returns (g(x), grad g(x))."""
        a, x, y = _f64(a), _f64(x), _f64(y)
        grad = np.empty(self.img_shape)
        val = _L().orc_g(self._s(), _ptr(a), _ptr(x), _ptr(y), _ptr(grad))
        return val, grad

    def r(self, b, a):
        """Returns (r(b), grad r(b))."""
        b, a = _f64(b), _f64(a)
        grad = np.empty(self.ker_shape)
        val = _L().orc_r(self._s(), _ptr(b), _ptr(a), _ptr(grad))
        return val, grad

    def upper(self, a, b, x, y):
        """Returns (ell = g(x) + r(b), ||grad_x ell||)."""
        gn = ct.c_double()
        val = _L().orc_upper(self._s(), _ptr(_f64(a)), _ptr(_f64(b)), _ptr(_f64(x)),
                             _ptr(_f64(y)), ct.byref(gn))
        return val, gn.value

    def hypergrad(self, a, b, x, y, delta, rhs=None, cg_max=1000, q0=None):
        """Returns (z, q, cg iterations, residual norm, capped)."""
        a, b, x, y = _f64(a), _f64(b), _f64(x), _f64(y)
        rp = None if rhs is None else _ptr(_f64(rhs))
        q = np.zeros(self.img_shape) if q0 is None else _f64(q0).copy()
        z = np.empty(self.ker_shape)
        res = ct.c_double()
        capped = ct.c_int()
        it = _L().orc_hypergrad(self._s(), _ptr(a), _ptr(b), _ptr(x), _ptr(y), rp, float(delta),
                                int(cg_max), _ptr(q), _ptr(z), ct.byref(res), ct.byref(capped))
        return z, q, it, res.value, bool(capped.value)

    def L_gx(self, a):
        return _L().orc_L_gx(self._s(), _ptr(_f64(a)))

    # ---------------------------------------------------------------- MAID
    def maid_init(self, a, **kw) -> MaidState:
        s = MaidState()
        _L().orc_maid_init(ct.byref(s))
        s.L_gx = self.L_gx(a)
        for k, v in kw.items():
            setattr(s, k, v)
        return s

    def maid_step(self, state: MaidState, a, y, b, x, q=None):
        """One upper iteration of Algorithm 2, in place on b, x (float64 arrays).
        Returns (accepted, q)."""
        assert b.dtype == np.float64 and x.dtype == np.float64
        q = np.zeros(self.img_shape) if q is None else q
        acc = _L().orc_maid_step(self._s(), ct.byref(state), _ptr(_f64(a)), _ptr(_f64(y)),
                                 _ptr(b), _ptr(x), _ptr(q))
        return bool(acc), q


def bf16_round(a) -> np.ndarray:
    """Operands of the BF16-input operator: each value rounded first to FP32,
    then to bfloat16 (1 sign, 8 exponent, 7 stored mantissa bits: FP32 with
    the low 16 bits dropped) with round-to-nearest, ties to even, returned as
    float64.  Written out on the FP32 bit pattern: add 0x7FFF plus the lowest
    kept bit, then clear the low 16 bits (finite inputs only)."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def norm(v) -> float:
    v = _f64(v).ravel()
    return _L().orc_norm(_ptr(v), v.size)
