"""Helpers shared by the GPU parity tests: build the same seeded instance for
the CUDA path (torch tensors) and for the FP64 oracle (NumPy float64 copies of
exactly the values the GPU sees)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_09758_gb300 import adp, synth


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_09758_gb300 import build
    build.build()


class Pair:
    """A problem on both sides.  dt: torch dtype of the GPU path."""

    def __init__(self, inst, prec=adp.ADP_F32, alpha=1e-2, reg=adp.ADP_REG_HUBER_TV, reg_param=1e-2,
                 beta=0.3, w0=1.0, timeout=2.0):
        C, H, W = inst.shape
        K = inst.K
        self.inst = inst
        self.dt = torch.float32 if prec == adp.ADP_F32 else torch.float64
        npdt = np.float32 if prec == adp.ADP_F32 else np.float64
        # the values both sides use (rounded once to the GPU's type)
        self.y = inst.y.astype(npdt).astype(np.float64)
        self.a = inst.a.astype(npdt).astype(np.float64)
        self.P = oracle.Problem(C, H, W, K, alpha=alpha, reg_param=reg_param, reg=reg, beta=beta, w0=w0)
        self.params = adp.Params(C, H, W, K, alpha=alpha, reg_param=reg_param, reg=reg, beta=beta,
                                 sobolev_w0=w0, prec=prec, wait_timeout_s=timeout)
        self.prob = adp.Problem(self.params, self.t(self.y), self.t(self.a))

    def t(self, arr):
        return torch.tensor(np.asarray(arr), dtype=self.dt, device="cuda").contiguous()

    def rounded(self, arr):
        """arr rounded to the GPU type, as float64 (what the oracle must see)."""
        return self.t(arr).double().cpu().numpy()

    @staticmethod
    def n(t):
        return t.detach().double().cpu().numpy()


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def psnr(x, ref, peak=1.0):
    mse = float(np.mean((np.asarray(x) - np.asarray(ref)) ** 2))
    return 10 * np.log10(peak ** 2 / mse)
