"""GPU parity of the 1D elastic-net variant (Sec. 4.1; cluster kernel in
csrc/adp_en1d.cu) against the FP64 oracle (oracle/en1d.py), through the C ABI.

Both sides see the same FP32-representable inputs.  The GPU computes in FP32
with FP64 dot products, norms and line-search tests, so:
* iteration-matched proximal-gradient iterates agree to 1e-5 relative and the
  gradient-mapping norm to 1e-5 relative plus 2e-6 (the Gram form's absolute
  rounding), eps-stopped solves stop within one iteration;
* the upper loss and its gradient norm agree to 1e-6;
* iteration-matched support CG (q) and the hypergradient z agree to 1e-4, and
  so does z from CG run to tolerance;
* MAID steps take the same decisions (acceptance, rounds, trials, eps, delta,
  step) with B and x within 1e-4;
* a device-resident run of several steps equals the same steps one launch at
  a time, bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import en1d
from paper_2502_09758_gb300 import adp, synth
from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


class Pair1D:
    def __init__(self, n, seed=0, perturb=0.0):
        s = synth.signal1d(n, seed=seed)
        f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        self.A = f32(s.A)
        self.y = f32(s.y)
        rng = np.random.default_rng(100 + seed)
        self.B = f32(s.A + perturb * rng.standard_normal((n, n)) / n)
        self.P = en1d.Problem(self.A, self.y)
        self.g = adp.En1d(self.t(self.A), self.t(self.y))
        self.n = n

    @staticmethod
    def t(a):
        return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()

    @staticmethod
    def h(t):
        return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,perturb", [(64, 0.0), (256, 0.0), (256, 0.5), (384, 0.2)])
def test_lower_solve_iteration_matched(n, perturb):
    pr = Pair1D(n, seed=1, perturb=perturb)
    for k in (1, 7, 60):
        xg = pr.t(pr.y)
        it, gn = pr.g.lower_solve(pr.t(pr.B), xg, 0.0, k)
        xo, ito, gno = pr.P.lower_solve(pr.B, pr.y, 0.0, k)
        assert it == ito == k
        assert rel(pr.h(xg), xo) <= 1e-5
        # the GPU forms grad f as (B^T B) x - B^T y: its rounding is absolute,
        # ~u ||B^T B|| ||x|| (about 5e-7 here), whatever the size of G
        assert abs(gn - gno) <= 1e-5 * gno + 2e-6


@pytest.mark.parametrize("eps", [1e-2, 1e-3])
def test_lower_solve_stops_like_the_oracle(eps):
    pr = Pair1D(256, seed=2)
    xg = pr.t(pr.y)
    it, gn = pr.g.lower_solve(pr.t(pr.B), xg, eps, 300)
    xo, ito, gno = pr.P.lower_solve(pr.B, pr.y, eps, 300)
    assert abs(it - ito) <= 1
    if it == ito:
        assert rel(pr.h(xg), xo) <= 1e-5
    assert gn <= eps or it == 300


def test_upper_loss():
    pr = Pair1D(256, seed=3)
    x = np.asarray(pr.y * 0.9, np.float32).astype(np.float64)
    l, g = pr.g.upper_loss(pr.t(x))
    lo, go = pr.P.upper(x)
    assert abs(l - lo) <= 1e-6 * lo and abs(g - go) <= 1e-6 * go


# (the CG of the 256 case meets 1e-5 after 32 iterations; beyond that the
# FP32 recurrences work on residuals at rounding level, and even a plain FP32
# CG on the CPU differs from FP64 by 1.0e-4 at 40 iterations)
@pytest.mark.parametrize("n,iters", [(64, 5), (256, 10), (256, 20)])
def test_hypergrad_iteration_matched(n, iters):
    pr = Pair1D(n, seed=4, perturb=0.3)
    xo, _, _ = pr.P.lower_solve(pr.B, pr.y, 1e-4, 2000)
    x = np.asarray(xo, np.float32).astype(np.float64)      # the same support on both sides
    assert 0 < (x != 0).sum() < n
    z, q, it, res = pr.g.hypergrad(pr.t(pr.B), pr.t(x), 0.0, iters)
    zo, qo, ito, reso, _ = pr.P.hypergrad(pr.B, x, 0.0, iters)
    assert it == ito == iters
    assert np.all(pr.h(q)[x == 0] == 0.0)
    assert rel(pr.h(q), qo) <= 1e-4
    assert rel(pr.h(z), zo) <= 1e-4
    assert abs(res - reso) <= 1e-3 * reso


@pytest.mark.parametrize("delta", [1e-3, 1e-5])
def test_hypergrad_to_tolerance(delta):
    """At delta = 1e-5 the FP32 recurrences approach their attainable accuracy
    and need a few more iterations than FP64 (34 against 30 here): the
    iteration count is compared at the looser delta only."""
    pr = Pair1D(256, seed=5, perturb=0.3)
    xo, _, _ = pr.P.lower_solve(pr.B, pr.y, 1e-4, 2000)
    x = np.asarray(xo, np.float32).astype(np.float64)
    z, q, it, res = pr.g.hypergrad(pr.t(pr.B), pr.t(x), delta, 1000)
    zo, qo, ito, reso, _ = pr.P.hypergrad(pr.B, x, delta, 1000)
    assert res <= delta
    if delta >= 1e-3:
        # a solve stopped at ||r|| ~ 3e-3 of ||rhs||: z carries that much
        # truncation, so the two sides agree to its rounding only loosely
        assert abs(it - ito) <= 1
        assert rel(pr.h(z), zo) <= 2e-4
    else:
        assert rel(pr.h(z), zo) <= 1e-4


def run_both(pr, steps, **over):
    sg = pr.g.maid_init(**over)
    so = pr.P.maid_init(**over)
    Bg, xg = pr.t(pr.B), pr.t(pr.y)
    Bo, xo = pr.B.copy(), pr.y.copy()
    for k in range(steps):
        acc_g = pr.g.maid_step(sg, Bg, xg)
        acc_o = pr.P.maid_step(so, Bo, xo)
        assert acc_g == acc_o, k
        assert (sg.rounds, sg.trials, sg.stopped) == (so.rounds, so.trials, so.stopped), k
        assert sg.eps == so.eps and sg.delta == so.delta and sg.step == so.step, k
        assert abs(sg.ll_iters - so.ll_iters) <= 2 * sg.trials + 2, k
    return sg, so, Bg, xg, Bo, xo


def test_maid_steps_match_the_oracle():
    pr = Pair1D(128, seed=6)
    sg, so, Bg, xg, Bo, xo = run_both(pr, 3, eps=1e-3, delta=1e-3, step=0.1)
    assert so.k >= 1
    assert rel(pr.h(Bg), Bo) <= 1e-4
    assert rel(pr.h(xg), xo) <= 1e-4
    assert abs(sg.loss - so.loss) <= 1e-4 * so.loss


def test_device_resident_run_equals_single_steps():
    pr = Pair1D(128, seed=7)
    over = dict(eps=1e-3, delta=1e-3, step=0.1)
    s1 = pr.g.maid_init(**over)
    B1, x1 = pr.t(pr.B), pr.t(pr.y)
    n1 = 0
    for _ in range(4):
        acc = pr.g.maid_step(s1, B1, x1)
        n1 += 1
        if not acc or s1.stopped:
            break
    s2 = pr.g.maid_init(**over)
    B2, x2 = pr.t(pr.B), pr.t(pr.y)
    n2 = pr.g.maid_run(s2, B2, x2, 4)
    assert n1 == n2
    assert torch.equal(B1, B2) and torch.equal(x1, x2)
    assert (s1.k, s1.eps, s1.step, s1.loss) == (s2.k, s2.eps, s2.step, s2.loss)


def test_invalid_sizes_are_rejected():
    y = torch.zeros(100, device="cuda")
    A = torch.zeros((100, 100), device="cuda")
    with pytest.raises(adp.AdpError):
        adp.En1d(A, y)                       # not a multiple of 32
    y = torch.zeros(392, device="cuda")
    A = torch.zeros((392, 392), device="cuda")
    with pytest.raises(adp.AdpError):
        adp.En1d(A, y)                       # above the maximum size
