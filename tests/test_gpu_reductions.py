"""Precision of the FP32 path's reductions (float-float combination of FP32
partial sums, standing in for the FP64 sums of the CG dot products, the norms
and the stopping tests).  An adversarial input: the gradient of h with a
delta kernel and alpha = 0 is x - y exactly, here one value 2^12 among
3 x 1024 x 1024 values 2^-6.  The small values carry 4.6e-5 of the squared
norm; a plain FP32 sum across threads would drop them all (2^-8-sized
partials against an ulp of 2 at 2^24).  The library's norm must agree with
the FP64 norm of the very gradient it returned to 1e-9 relative, on the
direct and on the FFT operator path."""
import numpy as np
import pytest
import torch

from paper_2502_09758_gb300 import adp
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("fft", [False, True])
def test_norm_reduction_keeps_small_terms(fft):
    C, H, W, K = 3, 1024, 1024, 1
    y = torch.zeros((C, H, W), dtype=torch.float32, device="cuda")
    a = torch.ones((C, K, K), dtype=torch.float32, device="cuda")
    prob = adp.Problem(adp.Params(C, H, W, K, alpha=0.0, reg_param=1e-2, beta=0.0), y, a)
    if fft:
        prob.set_fft(True)
    x = torch.full((C, H, W), 2.0 ** -6, dtype=torch.float32, device="cuda")
    x[1, 517, 300] = 2.0 ** 12
    g, nrm = prob.grad_lower(a, x)
    gd = g.double()
    exact = float((gd * gd).sum())
    if not fft:                            # the direct path returns x - y exactly here
        assert torch.equal(g, x)
        assert exact == 2.0 ** 24 + (C * H * W - 1) * 2.0 ** -12
    assert abs(nrm * nrm - exact) <= 1e-9 * exact
    # the small terms are resolved: without them the norm would be 2^12
    assert nrm * nrm - 2.0 ** 24 > 0.5 * (C * H * W - 1) * 2.0 ** -12
    prob.close()
