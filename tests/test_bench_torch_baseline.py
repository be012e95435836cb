"""The MAID written with PyTorch tensor ops (bench.py's second GPU baseline)
follows the same algorithm and readings as the oracle: run in FP64 on the CPU
on tiny problems it reproduces the oracle's MAID steps (same iteration counts,
same b and x to rounding)."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2502_09758_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("seed,fft", [(2, False), (3, False), (2, True), (4, True)])
def test_torch_maid_matches_oracle(seed, fft, monkeypatch):
    """Both operator forms of the PyTorch baseline: depthwise convolutions, and
    the convolution theorem through torch.fft (kernel wider than the image
    height included, so that wrapped taps add up)."""
    inst = synth.small(C=2, H=12, W=10, K=5, seed=seed) if seed != 4 else synth.small(C=1, H=4, W=8, K=5, seed=seed)
    monkeypatch.setattr(bench, "EPS0", 1e-4)
    monkeypatch.setattr(bench, "STEP0", 1e-3)
    monkeypatch.setattr(bench, "EPS_STOP", 0.0)
    _, fused, ups, b, x = bench.torch_maid_run(inst, 2, torch.float64, torch.device("cpu"), fft=fft)
    C, H, W = inst.shape
    P = oracle.Problem(C, H, W, inst.K, alpha=1e-2, reg_param=1e-2, beta=0.3)
    so = P.maid_init(inst.a, eps=1e-4, delta=1e-4, step=1e-3)
    bo, xo = inst.a.copy(), inst.y.copy()
    it, n = 0, 0
    for _ in range(2):
        acc, _ = P.maid_step(so, inst.a, inst.y, bo, xo)
        it += so.ll_iters + so.cg_iters
        n += 1
        if not acc:
            break
    assert ups == n and fused == it
    tol = 1e-10 if fft else 1e-12      # FFT rounding of the FP64 transforms
    assert np.linalg.norm(b.numpy() - bo) <= tol * np.linalg.norm(bo)
    assert np.linalg.norm(x.numpy() - xo) <= tol * np.linalg.norm(xo)
