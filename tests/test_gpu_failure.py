"""Failure detection without a GPU fault: a grid barrier that one CTA never
reaches makes the bounded waits of the others run out; the call must return
ADP_ETIMEOUT after about the problem's wait limit, and the same problem and
CUDA context must keep working afterwards."""
import time

import numpy as np
import pytest
import torch

from paper_2502_09758_gb300 import adp, synth
from gpu_common import Pair, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("prec", [adp.ADP_F32, adp.ADP_F64])
def test_bounded_wait_times_out_and_context_survives(prec):
    inst = synth.small(C=3, H=64, W=64, K=7, seed=1)
    limit = 0.1
    pr = Pair(inst, prec=prec, timeout=limit)
    assert pr.prob.grid_size() >= 2
    b, x = pr.t(pr.rounded(inst.b_true)), pr.t(pr.rounded(inst.x_true))
    before = pr.n(pr.prob.apply_B(b, x))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = pr.prob.selftest_wait_timeout()
    dt = time.perf_counter() - t0
    assert st == adp.ADP_ETIMEOUT, st
    assert limit * 0.9 <= dt <= 10.0, dt
    assert b"gave up" in adp.load_library().adp_last_error()
    # the context and the problem are still usable, with the same results
    after = pr.n(pr.prob.apply_B(b, x))
    assert rel(after, before) == 0.0
    it, gn, capped = pr.prob.lower_solve(b, x, 1e-3, 50)
    assert np.isfinite(gn) and it >= 1


def test_selftest_needs_two_ctas():
    inst = synth.small(C=1, H=8, W=8, K=3, seed=0)
    pr = Pair(inst, prec=adp.ADP_F32, timeout=0.1)
    if pr.prob.grid_size() >= 2:
        pytest.skip("this device launches more than one CTA for an 8x8 image")
    assert pr.prob.selftest_wait_timeout() == adp.ADP_EINVAL
