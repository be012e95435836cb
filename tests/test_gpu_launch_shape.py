"""The direct path's launch shape (adp_set_launch) and its autotuner
(runtime.choose_launch).  The shape only changes which warp takes which strip
and the order of the reduction sums, so results at any accepted shape match
the oracle within the parity tolerances; the autotuner keeps the shape it
measured fastest."""
import numpy as np
import pytest

from paper_2502_09758_gb300 import adp, runtime, synth
from gpu_common import Pair, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def gauss(C, H, W, K, seed=0):
    s = max(K / 5.0, 0.5)
    return synth.make_instance("l", C, H, W, synth.gaussian_kernel(K, 1.2 * s), synth.gaussian_kernel(K, s), 0.01, seed)


@pytest.mark.parametrize("prec,shapes", [(adp.ADP_F32, [(12, 4), (7, 2), (30, 8), (64, 6)]),
                                         (adp.ADP_F64, [(5, 2), (16, 4)])])
def test_results_hold_at_every_launch_shape(prec, shapes):
    C, H, W, K = (3, 70, 45, 7) if prec == adp.ADP_F32 else (1, 64, 64, 7)
    pr = Pair(gauss(C, H, W, K), prec=prec, beta=0.3)
    x0, b = pr.rounded(pr.inst.y), pr.rounded(pr.inst.a)
    xo, _, gno = pr.P.fista(b, pr.y, x0, eps=0.0, max_iters=15)
    rng = np.random.default_rng(1)
    v = pr.rounded(rng.standard_normal((C, H, W)))
    co = pr.P.cross_t(b, x0, pr.y, v)
    tol = 1e-5 if prec == adp.ADP_F32 else 1e-12
    for g, nw in shapes:
        pr.prob.set_launch(g, nw)
        assert (pr.prob.grid_size(), pr.prob.warps_per_cta()) == (g, nw)
        xg = pr.t(x0)
        it, gn, _ = pr.prob.lower_solve(pr.t(b), xg, eps=0.0, max_iters=15)
        assert it == 15 and rel(pr.n(xg), xo) <= tol, (g, nw)
        out = pr.prob.cross_t(pr.t(b), pr.t(x0), pr.t(v))
        assert rel(pr.n(out), co) <= (1e-6 if prec == adp.ADP_F32 else 1e-12), (g, nw)


def test_invalid_launch_shapes_are_rejected():
    pr = Pair(gauss(1, 32, 32, 5), prec=adp.ADP_F32)
    for g, nw in [(8, 3), (8, 10), (0, 8), (513, 8), (100000, 8)]:
        with pytest.raises(adp.AdpError) as e:
            pr.prob.set_launch(g, nw)
        assert e.value.status == adp.ADP_EINVAL
    # the problem stays usable at its shape
    x = pr.t(pr.rounded(pr.inst.y))
    pr.prob.lower_solve(pr.t(pr.rounded(pr.inst.a)), x, eps=1e-1)


def test_choose_launch_keeps_the_fastest_and_stays_exact():
    C, H, W, K = 3, 256, 256, 15
    inst = synth.make_instance("m", C, H, W, synth.motion_kernel(K, 11, 30), synth.motion_kernel(K, 11, 20), 0.02, 0)
    pr = Pair(inst, prec=adp.ADP_F32, beta=0.3)
    x0, b = pr.rounded(inst.y), pr.rounded(inst.a)
    res = runtime.choose_launch(pr.prob, pr.t(b), pr.t(x0), iters=8, reps=1)
    assert res["ms"] and min(res["ms"], key=res["ms"].get) == (res["grid"], res["nw"])
    assert (pr.prob.grid_size(), pr.prob.warps_per_cta()) == (res["grid"], res["nw"])
    xg = pr.t(x0)
    pr.prob.lower_solve(pr.t(b), xg, eps=0.0, max_iters=4)
    xo, _, _ = pr.P.fista(b, pr.y, x0, eps=0.0, max_iters=4)
    assert rel(pr.n(xg), xo) <= 1e-5
