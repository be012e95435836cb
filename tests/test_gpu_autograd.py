"""The differentiable lower-level solution x~(b) (torch.autograd.Function whose
backward is the IFT adjoint CG of Eq. 3.2, through adp_hypergrad with an
explicit right-hand side), checked against central finite differences of the
forward solve and against the FP64 oracle's hypergradient.

Scalar test function: L(b) = <w, x~(b)> for a fixed seeded w, so that
dL/db = -(grad^2_{xb} h)^T (grad^2_x h)^{-1} w.
"""
import numpy as np
import pytest
import torch

from paper_2502_09758_gb300 import adp, synth
from gpu_common import Pair, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _pair(prec, reg=adp.ADP_REG_SQRT_TV, reg_param=0.1):
    inst = synth.small(C=2, H=16, W=20, K=5, seed=3, sigma_true=1.0, sigma_init=0.8)
    return Pair(inst, prec=prec, alpha=1e-2, reg=reg, reg_param=reg_param)


def test_autograd_backward_matches_finite_differences_and_oracle():
    """FP64: autograd gradient vs central differences of L along random
    directions (solves to 1e-12, step 1e-4; the bound covers
    the O(h^2) truncation and the solve error over h) and vs the oracle's z with rhs = w."""
    pr = _pair(adp.ADP_F64)
    C, H, W = pr.inst.shape
    K = pr.inst.K
    rng = np.random.default_rng(7)
    w = rng.standard_normal((C, H, W))
    b0 = pr.rounded(pr.inst.a)
    eps, iters = 1e-12, 60000

    b = pr.t(b0).requires_grad_(True)
    x = adp.lower_solution(b, pr.prob, pr.t(pr.y), eps, 1e-13, max_iters=iters, cg_max_iters=5000)
    L = (x * pr.t(w)).sum()
    L.backward()
    g = pr.n(b.grad)
    assert np.all(np.isfinite(g))

    def L_at(bv):
        xv = pr.t(pr.y)
        pr.prob.lower_solve(pr.t(bv), xv, eps, iters)
        return float((pr.n(xv) * w).sum())

    h = 1e-4
    for k in range(3):
        d = rng.standard_normal((C, K, K))
        fd = (L_at(b0 + h * d) - L_at(b0 - h * d)) / (2 * h)
        an = float((g * d).sum())
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (k, fd, an)

    # the oracle's hypergradient with the same right-hand side at its own x~(b)
    xo, _, _ = pr.P.fista(b0, pr.y, pr.y, eps, iters)
    zo, _, _, _, _ = pr.P.hypergrad(pr.a, b0, xo, pr.y, 1e-13, rhs=w, cg_max=5000)
    assert rel(g, zo) <= 1e-7, rel(g, zo)


def test_autograd_fp32_matches_oracle():
    """FP32 forward and backward against the FP64 oracle, iteration-matched
    (30 FISTA updates, 10 CG iterations); the oracle's backward is taken at the
    GPU's x~ so that only the backward's own rounding is compared."""
    pr = _pair(adp.ADP_F32)
    C, H, W = pr.inst.shape
    rng = np.random.default_rng(11)
    w = pr.rounded(rng.standard_normal((C, H, W)))
    b0 = pr.rounded(pr.inst.a)
    b = pr.t(b0).requires_grad_(True)
    x = adp.lower_solution(b, pr.prob, pr.t(pr.y), 0.0, 0.0, max_iters=30, cg_max_iters=10)
    (x * pr.t(w)).sum().backward()
    xo, ito, _ = pr.P.fista(b0, pr.y, pr.y, 0.0, 30)
    assert ito == 30
    assert rel(pr.n(x), xo) <= 1e-5
    zo, _, _, _, _ = pr.P.hypergrad(pr.a, b0, pr.n(x), pr.y, 0.0, rhs=w, cg_max=10)
    assert rel(pr.n(b.grad), zo) <= 1e-4, rel(pr.n(b.grad), zo)


def test_autograd_composes_with_a_torch_loss():
    """grad of a torch-side loss of x~(b) flows back to b and agrees with the
    hypergradient called directly with rhs = dloss/dx."""
    pr = _pair(adp.ADP_F64, reg=adp.ADP_REG_HUBER_TV, reg_param=1e-2)
    b = pr.t(pr.rounded(pr.inst.a)).requires_grad_(True)
    target = pr.t(pr.inst.x_true)
    x = adp.lower_solution(b, pr.prob, pr.t(pr.y), 1e-11, 1e-12, max_iters=60000, cg_max_iters=5000)
    loss = ((x - target) ** 2).sum()
    loss.backward()
    gx = (2 * (x.detach() - target)).contiguous()
    z, _, _, _, _ = pr.prob.hypergrad(b.detach(), x.detach(), 1e-12, rhs=gx, max_iters=5000)
    assert rel(pr.n(b.grad), pr.n(z)) <= 1e-12
