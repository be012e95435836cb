"""ctypes binding of libadp.so (C ABI in include/adp.h).

Argument marshalling only: every step of the hot path runs in the CUDA kernels
of libadp.  Tensors are PyTorch CUDA tensors (device memory, streams); they
are checked for device, dtype, shape and contiguity and passed as raw device
pointers.  There is no CPU path: if the library or a GPU is missing, loading
raises.

The functions carry the C names (``adp_lower_solve`` ...); :class:`Problem`
wraps them for convenience.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libadp.so")

ADP_OK, ADP_EINVAL, ADP_ENOMEM, ADP_ECUDA, ADP_ENONFINITE, ADP_ENOCONV, ADP_ELSFAIL, ADP_ETIMEOUT = range(8)
ADP_F64, ADP_F32 = 0, 1
ADP_REG_HUBER_TV, ADP_REG_SQRT_TV, ADP_REG_QUAD = 0, 1, 2

# every entry point declared in include/adp.h
EXPORTS = ("adp_problem_create", "adp_problem_destroy", "adp_apply_B", "adp_apply_Bt",
           "adp_apply_B_bf16", "adp_apply_Bt_bf16", "adp_bf16_prep_ms_last", "adp_bf16_grid_size",
           "adp_set_fft", "adp_fft_enabled", "adp_fft_pipeline", "adp_set_launch",
           "adp_grad_lower", "adp_hess_vec", "adp_lower_solve", "adp_upper_loss", "adp_hypergrad",
           "adp_cross_t", "adp_maid_init", "adp_maid_step", "adp_conv_passes_last",
           "adp_grid_size", "adp_warps_per_cta", "adp_last_kernel_ms", "adp_trace_enable",
           "adp_trace_read", "adp_lower_solve_noalloc", "adp_selftest_wait_timeout", "adp_batch_create",
           "adp_batch_destroy", "adp_batch_maid_step", "adp_batch_maid_run_graph", "adp_batch_group_size",
           "adp_batch_last_kernel_ms", "adp_last_error", "adp_status_string",
           "adp_en1d_create", "adp_en1d_destroy", "adp_en1d_lower_solve", "adp_en1d_upper_loss",
           "adp_en1d_hypergrad", "adp_en1d_maid_init", "adp_en1d_maid_step", "adp_en1d_maid_run")


class AdpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"adp status {status}: {msg}")
        self.status = status


class adp_params(ct.Structure):
    _fields_ = [("C", ct.c_int), ("H", ct.c_int), ("W", ct.c_int), ("K", ct.c_int),
                ("alpha", ct.c_double), ("reg_param", ct.c_double), ("reg", ct.c_int),
                ("beta", ct.c_double), ("sobolev_w0", ct.c_double), ("prec", ct.c_int),
                ("wait_timeout_s", ct.c_double)]


class adp_en1d_params(ct.Structure):
    _fields_ = [("n", ct.c_int), ("a1", ct.c_double), ("a2", ct.c_double), ("lam", ct.c_double)]


class adp_maid_state(ct.Structure):
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


_lib = None


def load_library(path: str = LIB_PATH) -> ct.CDLL:
    """Load libadp.so (no fallback: raises when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libadp.so not built at {path}; run __graft_entry__.build() "
                               "or python -m paper_2502_09758_gb300.build")
        lib = ct.CDLL(path)
        P, vp, d, i = ct.c_void_p, ct.c_void_p, ct.c_double, ct.c_int
        dp, ip = ct.POINTER(ct.c_double), ct.POINTER(ct.c_int)
        sig = {
            "adp_problem_create": (i, [ct.POINTER(adp_params), vp, vp, vp, ct.POINTER(ct.c_void_p)]),
            "adp_problem_destroy": (None, [P]),
            "adp_apply_B": (i, [P, vp, vp, vp]),
            "adp_apply_Bt": (i, [P, vp, vp, vp]),
            "adp_apply_B_bf16": (i, [P, vp, vp, vp]),
            "adp_apply_Bt_bf16": (i, [P, vp, vp, vp]),
            "adp_bf16_prep_ms_last": (ct.c_double, [P]),
            "adp_bf16_grid_size": (i, [P]),
            "adp_set_fft": (i, [P, i]),
            "adp_fft_enabled": (i, [P]),
            "adp_fft_pipeline": (i, [P]),
            "adp_set_launch": (i, [P, i, i]),
            "adp_grad_lower": (i, [P, vp, vp, vp, dp]),
            "adp_hess_vec": (i, [P, vp, vp, vp, vp]),
            "adp_lower_solve": (i, [P, vp, vp, d, i, ip, dp]),
            "adp_upper_loss": (i, [P, vp, vp, dp, dp, vp]),
            "adp_hypergrad": (i, [P, vp, vp, vp, d, i, vp, vp, ip, dp]),
            "adp_cross_t": (i, [P, vp, vp, vp, vp]),
            "adp_maid_init": (i, [P, ct.POINTER(adp_maid_state)]),
            "adp_maid_step": (i, [P, ct.POINTER(adp_maid_state), vp, vp, vp]),
            "adp_conv_passes_last": (ct.c_longlong, [P]),
            "adp_grid_size": (i, [P]),
            "adp_warps_per_cta": (i, [P]),
            "adp_last_kernel_ms": (ct.c_double, [P]),
            "adp_trace_enable": (i, [P, i]),
            "adp_trace_read": (i, [P, ct.POINTER(ct.c_longlong), i]),
            "adp_lower_solve_noalloc": (i, [ct.POINTER(adp_params), vp, vp, vp, d, i, vp, ip, dp]),
            "adp_selftest_wait_timeout": (i, [P]),
            "adp_batch_create": (i, [ct.POINTER(ct.c_void_p), i, ct.POINTER(ct.c_void_p)]),
            "adp_batch_destroy": (None, [P]),
            "adp_batch_maid_step": (i, [P, ct.POINTER(adp_maid_state), ct.POINTER(ct.c_void_p),
                                        ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_void_p)]),
            "adp_batch_maid_run_graph": (i, [P, ct.POINTER(adp_maid_state), ct.POINTER(ct.c_void_p),
                                             ct.POINTER(ct.c_void_p), ct.POINTER(ct.c_void_p), i,
                                             ct.POINTER(ct.c_longlong)]),
            "adp_batch_group_size": (i, [P, i]),
            "adp_batch_last_kernel_ms": (ct.c_double, [P]),
            "adp_last_error": (ct.c_char_p, []),
            "adp_status_string": (ct.c_char_p, [i]),
            "adp_en1d_create": (i, [ct.POINTER(adp_en1d_params), vp, vp, vp, ct.POINTER(ct.c_void_p)]),
            "adp_en1d_destroy": (None, [P]),
            "adp_en1d_lower_solve": (i, [P, vp, vp, d, i, ip, dp]),
            "adp_en1d_upper_loss": (i, [P, vp, dp, dp]),
            "adp_en1d_hypergrad": (i, [P, vp, vp, d, i, vp, vp, ip, dp]),
            "adp_en1d_maid_init": (i, [P, ct.POINTER(adp_maid_state)]),
            "adp_en1d_maid_step": (i, [P, ct.POINTER(adp_maid_state), vp, vp]),
            "adp_en1d_maid_run": (i, [P, ct.POINTER(adp_maid_state), vp, vp, i, ip]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(st, ok=(ADP_OK,)):
    if st not in ok:
        raise AdpError(st, load_library().adp_last_error().decode())
    return st


@dataclass
class Params:
    C: int
    H: int
    W: int
    K: int
    alpha: float = 1e-2
    reg_param: float = 1e-2
    reg: int = ADP_REG_HUBER_TV
    beta: float = 0.3
    sobolev_w0: float = 1.0
    prec: int = ADP_F32
    wait_timeout_s: float = 2.0

    def c(self) -> adp_params:
        return adp_params(self.C, self.H, self.W, self.K, self.alpha, self.reg_param, self.reg,
                          self.beta, self.sobolev_w0, self.prec, self.wait_timeout_s)

    @property
    def dtype(self):
        return torch.float32 if self.prec == ADP_F32 else torch.float64


def _ptr(t, shape, dtype, name, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ct.c_void_p(t.data_ptr())


# ------------------------------------------------------------- C-named calls
def adp_problem_create(params: Params, y: torch.Tensor, a: torch.Tensor, stream=None):
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream(y.device)
    handle = ct.c_void_p()
    cp = params.c()
    img, ker = (params.C, params.H, params.W), (params.C, params.K, params.K)
    with torch.cuda.device(y.device):
        _check(lib.adp_problem_create(ct.byref(cp), _ptr(y, img, params.dtype, "y"),
                                      _ptr(a, ker, params.dtype, "a"), ct.c_void_p(s.cuda_stream),
                                      ct.byref(handle)))
    return handle


def adp_problem_destroy(handle):
    load_library().adp_problem_destroy(handle)


class Problem:
    """One ADP-beta instance on one GPU (Eq. 2.5), owning the library handle."""

    def __init__(self, params: Params, y: torch.Tensor, a: torch.Tensor, stream=None):
        self.params = params
        self.device = y.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(y.device)
        self.handle = adp_problem_create(params, y, a, self.stream)
        self.lib = load_library()
        self.img = (params.C, params.H, params.W)
        self.ker = (params.C, params.K, params.K)
        self.dtype = params.dtype

    def close(self):
        if self.handle is not None:
            adp_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _i(self, t, name, optional=False):
        return _ptr(t, self.img, self.dtype, name, optional)

    def _k(self, t, name, optional=False):
        return _ptr(t, self.ker, self.dtype, name, optional)

    def _new_img(self):
        return torch.empty(self.img, dtype=self.dtype, device=self.device)

    # --------------------------------------------------------------- calls
    def apply_B(self, b, x, out=None):
        out = self._new_img() if out is None else out
        _check(self.lib.adp_apply_B(self.handle, self._k(b, "b"), self._i(x, "x"), self._i(out, "out")))
        return out

    def apply_Bt(self, b, z, out=None):
        out = self._new_img() if out is None else out
        _check(self.lib.adp_apply_Bt(self.handle, self._k(b, "b"), self._i(z, "z"), self._i(out, "out")))
        return out

    def apply_B_bf16(self, b, x, out=None):
        """B x with BF16 operands and FP32 accumulation (tensor cores); FP32 problems, K <= 33."""
        out = self._new_img() if out is None else out
        _check(self.lib.adp_apply_B_bf16(self.handle, self._k(b, "b"), self._i(x, "x"), self._i(out, "out")))
        return out

    def apply_Bt_bf16(self, b, z, out=None):
        """B^T z with BF16 operands and FP32 accumulation (tensor cores)."""
        out = self._new_img() if out is None else out
        _check(self.lib.adp_apply_Bt_bf16(self.handle, self._k(b, "b"), self._i(z, "z"), self._i(out, "out")))
        return out

    def set_fft(self, enable=True, complex_only=False):
        """Evaluate the operators of later calls through 2-D FFTs (FP32, power-of-two H, W);
        complex_only keeps the lower solves and CG off the real-to-complex pipeline."""
        _check(self.lib.adp_set_fft(self.handle, (2 if complex_only else 1) if enable else 0))

    def fft_enabled(self) -> bool:
        return bool(self.lib.adp_fft_enabled(self.handle))

    def set_launch(self, grid, nw):
        """Launch shape of the direct-path kernel: grid CTAs of nw warps."""
        _check(self.lib.adp_set_launch(self.handle, int(grid), int(nw)))

    def fft_pipeline(self) -> int:
        """0: direct correlation; 1: complex FFT pipeline; 2: real-to-complex lower solves."""
        return int(self.lib.adp_fft_pipeline(self.handle))

    def bf16_prep_ms(self) -> float:
        return float(self.lib.adp_bf16_prep_ms_last(self.handle))

    def bf16_grid_size(self) -> int:
        return int(self.lib.adp_bf16_grid_size(self.handle))

    def grad_lower(self, b, x, out=None):
        out = self._new_img() if out is None else out
        nrm = ct.c_double()
        _check(self.lib.adp_grad_lower(self.handle, self._k(b, "b"), self._i(x, "x"), self._i(out, "out"),
                                       ct.byref(nrm)))
        return out, nrm.value

    def hess_vec(self, b, x, v, out=None):
        out = self._new_img() if out is None else out
        _check(self.lib.adp_hess_vec(self.handle, self._k(b, "b"), self._i(x, "x"), self._i(v, "v"),
                                     self._i(out, "out")))
        return out

    def lower_solve(self, b, x, eps, max_iters=300):
        """In place on x; returns (updates, ||grad_x h||, capped)."""
        it, gn = ct.c_int(), ct.c_double()
        st = _check(self.lib.adp_lower_solve(self.handle, self._k(b, "b"), self._i(x, "x"), float(eps),
                                             int(max_iters), ct.byref(it), ct.byref(gn)),
                    ok=(ADP_OK, ADP_ENOCONV))
        return it.value, gn.value, st == ADP_ENOCONV

    def upper_loss(self, b, x, gradx=None):
        loss, gn = ct.c_double(), ct.c_double()
        _check(self.lib.adp_upper_loss(self.handle, self._k(b, "b"), self._i(x, "x"), ct.byref(loss),
                                       ct.byref(gn), self._i(gradx, "gradx", optional=True)))
        return loss.value, gn.value

    def hypergrad(self, b, x, delta, q=None, z=None, rhs=None, max_iters=1000):
        """Returns (z, q, cg iterations, residual norm, capped); q in/out (zeros if None)."""
        q = torch.zeros(self.img, dtype=self.dtype, device=self.device) if q is None else q
        z = torch.empty(self.ker, dtype=self.dtype, device=self.device) if z is None else z
        it, res = ct.c_int(), ct.c_double()
        st = _check(self.lib.adp_hypergrad(self.handle, self._k(b, "b"), self._i(x, "x"),
                                           self._i(rhs, "rhs", optional=True), float(delta), int(max_iters),
                                           self._i(q, "q"), self._k(z, "z"), ct.byref(it), ct.byref(res)),
                    ok=(ADP_OK, ADP_ENOCONV))
        return z, q, it.value, res.value, st == ADP_ENOCONV

    def cross_t(self, b, x, v, out=None):
        out = torch.empty(self.ker, dtype=self.dtype, device=self.device) if out is None else out
        _check(self.lib.adp_cross_t(self.handle, self._k(b, "b"), self._i(x, "x"), self._i(v, "v"),
                                    self._k(out, "out")))
        return out

    def maid_init(self, **overrides) -> adp_maid_state:
        s = adp_maid_state()
        _check(self.lib.adp_maid_init(self.handle, ct.byref(s)))
        for k, v in overrides.items():
            setattr(s, k, v)
        return s

    def maid_step(self, state: adp_maid_state, b, x, q):
        """One upper iteration of Algorithm 2 in place on b, x, q; returns
        accepted (False also when the stop rule fired: see state.stopped)."""
        st = _check(self.lib.adp_maid_step(self.handle, ct.byref(state), self._k(b, "b"), self._i(x, "x"),
                                           self._i(q, "q")), ok=(ADP_OK, ADP_ELSFAIL))
        return st == ADP_OK and bool(state.accepted)

    def conv_passes_last(self) -> int:
        return int(self.lib.adp_conv_passes_last(self.handle))

    def grid_size(self) -> int:
        return int(self.lib.adp_grid_size(self.handle))

    def warps_per_cta(self) -> int:
        return int(self.lib.adp_warps_per_cta(self.handle))

    def last_kernel_ms(self) -> float:
        return float(self.lib.adp_last_kernel_ms(self.handle))

    def selftest_wait_timeout(self) -> int:
        """Run the failure-path diagnostic (a grid barrier CTA 0 never reaches);
        returns the raw status, ADP_ETIMEOUT when the bounded waits work."""
        return int(self.lib.adp_selftest_wait_timeout(self.handle))

    def trace_enable(self, cap: int):
        _check(self.lib.adp_trace_enable(self.handle, int(cap)))
        self._trace_cap = int(cap)

    def trace_read(self):
        """(arrive, leave) global-timer pairs (ns) of CTA 0 for the last call."""
        import numpy as np
        cap = getattr(self, "_trace_cap", 0)
        buf = (ct.c_longlong * (2 * max(cap, 1)))()
        n = self.lib.adp_trace_read(self.handle, buf, cap)
        return np.array(buf[: 2 * max(n, 0)], dtype=np.int64).reshape(-1, 2)


def adp_lower_solve(prob: Problem, b, x, eps, max_iters=300):
    return prob.lower_solve(b, x, eps, max_iters)


def adp_hypergrad(prob: Problem, b, x, delta, q=None, z=None, rhs=None, max_iters=1000):
    return prob.hypergrad(b, x, delta, q, z, rhs, max_iters)


def adp_upper_loss(prob: Problem, b, x, gradx=None):
    return prob.upper_loss(b, x, gradx)


def adp_maid_step(prob: Problem, state, b, x, q):
    return prob.maid_step(state, b, x, q)


def adp_maid_init(prob: Problem, **overrides):
    return prob.maid_init(**overrides)


def adp_lower_solve_noalloc(params: Params, y, b, x, eps, max_iters=300, stream=None):
    """adp_lower_solve without any device allocation (workspace in a fixed
    library array): for callers that cannot allocate device memory where they
    need the solve.  In place on x; returns (updates, ||grad_x h||, capped)."""
    lib = load_library()
    img, ker = (params.C, params.H, params.W), (params.C, params.K, params.K)
    for name, t in (("y", y), ("b", b)):
        if isinstance(t, torch.Tensor) and t.device != x.device:
            raise ValueError(f"{name} must be on {x.device}, got {t.device}")
    it, gn = ct.c_int(), ct.c_double()
    cp = params.c()
    # the library resolves its array and device limits for the current device
    with torch.cuda.device(x.device):
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        st = _check(lib.adp_lower_solve_noalloc(ct.byref(cp), _ptr(y, img, params.dtype, "y"),
                                                _ptr(b, ker, params.dtype, "b"), _ptr(x, img, params.dtype, "x"),
                                                float(eps), int(max_iters), ct.c_void_p(s.cuda_stream),
                                                ct.byref(it), ct.byref(gn)), ok=(ADP_OK, ADP_ENOCONV))
    return it.value, gn.value, st == ADP_ENOCONV


# ----------------------------------------------------------------- batches
class Batch:
    """Many problems in one cooperative launch (adp_batch_*): one MAID upper
    iteration of every problem per launch, or a whole device-resident run
    replayed from a CUDA graph.  The problems must outlive the batch."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.lib = load_library()
        self.n = len(self.problems)
        arr = (ct.c_void_p * self.n)(*[p.handle for p in self.problems])
        h = ct.c_void_p()
        with torch.cuda.device(self.problems[0].device):
            _check(self.lib.adp_batch_create(arr, self.n, ct.byref(h)))
        self.handle = h

    def close(self):
        if self.handle is not None:
            self.lib.adp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arrays(self, states, bs, xs, qs):
        st = (adp_maid_state * self.n)(*states)
        pb = (ct.c_void_p * self.n)(*[p._k(b, "b").value for p, b in zip(self.problems, bs)])
        px = (ct.c_void_p * self.n)(*[p._i(x, "x").value for p, x in zip(self.problems, xs)])
        pq = (ct.c_void_p * self.n)(*[p._i(q, "q").value for p, q in zip(self.problems, qs)])
        return st, pb, px, pq

    def maid_step(self, states, bs, xs, qs):
        """One upper iteration on every problem (in place); states are updated.
        Returns the list of accepted flags."""
        st, pb, px, pq = self._arrays(states, bs, xs, qs)
        _check(self.lib.adp_batch_maid_step(self.handle, st, pb, px, pq), ok=(ADP_OK, ADP_ELSFAIL))
        for i in range(self.n):
            ct.memmove(ct.byref(states[i]), ct.byref(st[i]), ct.sizeof(adp_maid_state))
        return [bool(s.accepted) for s in states]

    def maid_run_graph(self, states, bs, xs, qs, max_steps):
        """Up to max_steps upper iterations on every problem from one CUDA
        graph (state kept on the device).  Returns per-problem totals
        (fused iterations, convolution passes, upper iterations, accepted)."""
        st, pb, px, pq = self._arrays(states, bs, xs, qs)
        tot = (ct.c_longlong * (4 * self.n))()
        _check(self.lib.adp_batch_maid_run_graph(self.handle, st, pb, px, pq, int(max_steps), tot))
        for i in range(self.n):
            ct.memmove(ct.byref(states[i]), ct.byref(st[i]), ct.sizeof(adp_maid_state))
        return [tuple(tot[4 * i: 4 * i + 4]) for i in range(self.n)]

    def group_sizes(self):
        return [int(self.lib.adp_batch_group_size(self.handle, i)) for i in range(self.n)]

    def last_kernel_ms(self) -> float:
        return float(self.lib.adp_batch_last_kernel_ms(self.handle))


# ----------------------------------------------------------------- autograd
class En1d:
    """The 1D elastic-net variant of Sec. 4.1 on one GPU: the forward matrix
    A (n x n) and the data y (n), FP32 CUDA tensors; the learned operator B is
    a full n x n matrix passed to each call."""

    def __init__(self, A: torch.Tensor, y: torch.Tensor, a1=1.2e-3, a2=4e-3, lam=0.1, stream=None):
        n = y.shape[0]
        self.n, self.device = n, y.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(y.device)
        self.lib = load_library()
        self._A, self._y = A, y          # the library reads them at every call
        prm = adp_en1d_params(n, a1, a2, lam)
        h = ct.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.adp_en1d_create(ct.byref(prm), _ptr(A, (n, n), torch.float32, "A"),
                                            _ptr(y, (n,), torch.float32, "y"),
                                            ct.c_void_p(self.stream.cuda_stream), ct.byref(h)))
        self.handle = h

    def close(self):
        if self.handle is not None:
            self.lib.adp_en1d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _m(self, t, name):
        return _ptr(t, (self.n, self.n), torch.float32, name)

    def _v(self, t, name):
        return _ptr(t, (self.n,), torch.float32, name)

    def lower_solve(self, B, x, eps, max_iters=300):
        """x in/out; returns (updates, ||G||)."""
        it, gn = ct.c_int(), ct.c_double()
        with torch.cuda.device(self.device):
            _check(self.lib.adp_en1d_lower_solve(self.handle, self._m(B, "B"), self._v(x, "x"), eps, max_iters,
                                                 ct.byref(it), ct.byref(gn)))
        return it.value, gn.value

    def upper_loss(self, x):
        l, g = ct.c_double(), ct.c_double()
        with torch.cuda.device(self.device):
            _check(self.lib.adp_en1d_upper_loss(self.handle, self._v(x, "x"), ct.byref(l), ct.byref(g)))
        return l.value, g.value

    def hypergrad(self, B, x, delta, max_iters=1000):
        """Returns (z, q, CG iterations, ||r||)."""
        q = torch.empty(self.n, dtype=torch.float32, device=self.device)
        z = torch.empty((self.n, self.n), dtype=torch.float32, device=self.device)
        it, res = ct.c_int(), ct.c_double()
        with torch.cuda.device(self.device):
            _check(self.lib.adp_en1d_hypergrad(self.handle, self._m(B, "B"), self._v(x, "x"), delta, max_iters,
                                               self._v(q, "q"), self._m(z, "z"), ct.byref(it), ct.byref(res)))
        return z, q, it.value, res.value

    def maid_init(self, **overrides) -> adp_maid_state:
        s = adp_maid_state()
        _check(self.lib.adp_en1d_maid_init(self.handle, ct.byref(s)))
        for k, v in overrides.items():
            setattr(s, k, v)
        return s

    def maid_step(self, s, B, x) -> bool:
        with torch.cuda.device(self.device):
            _check(self.lib.adp_en1d_maid_step(self.handle, ct.byref(s), self._m(B, "B"), self._v(x, "x")))
        return bool(s.accepted)

    def maid_run(self, s, B, x, max_steps):
        steps = ct.c_int()
        with torch.cuda.device(self.device):
            _check(self.lib.adp_en1d_maid_run(self.handle, ct.byref(s), self._m(B, "B"), self._v(x, "x"),
                                              max_steps, ct.byref(steps)))
        return steps.value


class ADPLower(torch.autograd.Function):
    """x~(b): the lower-level solution as a differentiable function of the kernel.

    forward runs FISTA from the warm start ``x0`` (no iterates are stored; x~ is
    saved as the linearisation point).  backward is the IFT adjoint of Eq. 3.2:
    CG on grad^2_x h q = grad_output, then -(grad^2_{xb} h)^T q, computed by
    ``adp_hypergrad`` with an explicit right-hand side (no Sobolev term).
    """

    @staticmethod
    def forward(ctx, b, prob: Problem, x0, eps, delta, max_iters=300, cg_max_iters=1000):
        x = x0.detach().clone()
        prob.lower_solve(b.detach(), x, eps, max_iters)
        ctx.prob, ctx.delta, ctx.cg_max = prob, delta, cg_max_iters
        ctx.save_for_backward(b.detach(), x)
        return x

    @staticmethod
    def backward(ctx, gx):
        b, x = ctx.saved_tensors
        z, _, _, _, _ = ctx.prob.hypergrad(b, x, ctx.delta, rhs=gx.contiguous(), max_iters=ctx.cg_max)
        return z, None, None, None, None, None, None


def lower_solution(b, prob: Problem, x0, eps, delta=None, max_iters=300, cg_max_iters=1000):
    """Differentiable x~(b) (see :class:`ADPLower`); delta defaults to eps (Sec. 4.2)."""
    return ADPLower.apply(b, prob, x0, eps, eps if delta is None else delta, max_iters, cg_max_iters)
