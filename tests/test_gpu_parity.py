"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on the
same seeded inputs, row by row of the hot path.

Tolerances (written here, derived in the design notes):
  * operators (B, B^T, grad_x h, Hessian-vector, cross term) in FP32: relative L2 <= 1e-6 (2e-6
    for the two-pass compositions)
  * grad g = 2 A^T (A x - y): relative L2 <= max(2e-6, 8 u ||A x|| / ||A x - y||), the FP32
    rounding of the data residual amplified by its cancellation (u = 2^-24)
  * FP64 path: relative L2 <= 1e-12
  * iteration-matched FISTA iterates in FP32: relative L2 <= 1e-5
  * hypergradient z at matched eps/delta: relative error <= 1e-4
  * MAID: identical accept/reject decisions and adaptive constants; kernel and
    image PSNR within 0.05 dB.
"""
import numpy as np
import pytest
import torch

from paper_2502_09758_gb300 import adp, synth
from gpu_common import Pair, need_gpu, psnr, rel

pytestmark = pytest.mark.gpu

OP_TOL = {adp.ADP_F32: 1e-6, adp.ADP_F64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def inst_for(C, H, W, K, seed=0, kind="gauss"):
    if kind == "motion":
        return synth.make_instance("t", C, H, W, synth.motion_kernel(K, max(K - 4, 1), 30),
                                   synth.motion_kernel(K, max(K - 4, 1), 20), 0.02, seed)
    s = max(K / 5.0, 0.5)
    return synth.make_instance("t", C, H, W, synth.gaussian_kernel(K, s * 1.2),
                               synth.gaussian_kernel(K, s), 0.01, seed)


OP_CASES = [
    (1, 16, 16, 3, adp.ADP_F32),
    (3, 70, 45, 7, adp.ADP_F32),      # ragged tiles in both directions
    (2, 33, 97, 15, adp.ADP_F32),
    (1, 40, 40, 1, adp.ADP_F32),      # K = 1
    (1, 8, 10, 9, adp.ADP_F32),       # kernel larger than the image: multiple wraps
    (1, 12, 14, 31, adp.ADP_F32),     # halo wider than the image: ghosts hold several periods
    (1, 64, 80, 31, adp.ADP_F32),
    (3, 256, 256, 15, adp.ADP_F32),   # full size of the 256^2 RGB workload
    (1, 64, 64, 7, adp.ADP_F64),      # the 64^2 FP64 workload
    (2, 21, 50, 5, adp.ADP_F64),
]


@pytest.mark.parametrize("C,H,W,K,prec", OP_CASES)
def test_operators_B_Bt(C, H, W, K, prec):
    pr = Pair(inst_for(C, H, W, K, kind="motion" if K >= 15 else "gauss"), prec=prec)
    rng = np.random.default_rng(C * H + K)
    x = pr.rounded(rng.uniform(size=(C, H, W)))
    b = pr.rounded(pr.inst.b_true)
    out = pr.prob.apply_B(pr.t(b), pr.t(x))
    assert rel(pr.n(out), pr.P.conv(b, x)) <= OP_TOL[prec]
    out = pr.prob.apply_Bt(pr.t(b), pr.t(x))
    assert rel(pr.n(out), pr.P.conv_adj(b, x)) <= OP_TOL[prec]


@pytest.mark.parametrize("C,H,W,K,prec", [c for c in OP_CASES if c[1] * c[2] <= 70 * 70 or c[3] == 15])
@pytest.mark.parametrize("reg,par", [(adp.ADP_REG_HUBER_TV, 1e-2), (adp.ADP_REG_SQRT_TV, 1e-2),
                                     (adp.ADP_REG_QUAD, 0.0)])
def test_grad_and_hessian_of_lower_level(C, H, W, K, prec, reg, par):
    pr = Pair(inst_for(C, H, W, K), prec=prec, reg=reg, reg_param=par if par else 1.0, alpha=0.05)
    rng = np.random.default_rng(7)
    x = pr.rounded(pr.inst.x_true + 0.05 * rng.standard_normal((C, H, W)))
    v = pr.rounded(rng.standard_normal((C, H, W)))
    b = pr.rounded(pr.inst.a)
    g, nrm = pr.prob.grad_lower(pr.t(b), pr.t(x))
    go = pr.P.grad_h(b, x, pr.y)
    assert rel(pr.n(g), go) <= OP_TOL[prec] * 2
    assert nrm == pytest.approx(np.linalg.norm(go), rel=OP_TOL[prec] * 2)
    hv = pr.prob.hess_vec(pr.t(b), pr.t(x), pr.t(v))
    assert rel(pr.n(hv), pr.P.hess_h_vec(b, x, v)) <= OP_TOL[prec] * 2


@pytest.mark.parametrize("C,H,W,K,prec,n", [(3, 70, 45, 7, adp.ADP_F32, 25), (1, 64, 64, 7, adp.ADP_F64, 40),
                                            (3, 256, 256, 15, adp.ADP_F32, 4)])
def test_lower_solve_iteration_matched(C, H, W, K, prec, n):
    pr = Pair(inst_for(C, H, W, K, kind="motion" if K >= 15 else "gauss"), prec=prec)
    x0 = pr.rounded(pr.inst.y)
    b = pr.rounded(pr.inst.a)
    xg = pr.t(x0)
    it, gn, capped = pr.prob.lower_solve(pr.t(b), xg, eps=0.0, max_iters=n)
    xo, ito, gno = pr.P.fista(b, pr.y, x0, eps=0.0, max_iters=n)
    assert it == ito == n and capped
    tol = 1e-5 if prec == adp.ADP_F32 else 1e-12
    assert rel(pr.n(xg), xo) <= tol
    assert gn == pytest.approx(gno, rel=tol * 10)


@pytest.mark.parametrize("eps", [1e-1, 2e-2])
def test_lower_solve_stop_rule(eps):
    pr = Pair(inst_for(3, 70, 45, 7), prec=adp.ADP_F32)
    x0, b = pr.rounded(pr.inst.y), pr.rounded(pr.inst.a)
    xg = pr.t(x0)
    k, gn, capped = pr.prob.lower_solve(pr.t(b), xg, eps=eps, max_iters=300)
    assert not capped and gn <= eps and k > 0
    # the oracle agrees that the test passes at k and not at k - 1
    _, _, g_k = pr.P.fista(b, pr.y, x0, eps=0.0, max_iters=k)
    _, _, g_km1 = pr.P.fista(b, pr.y, x0, eps=0.0, max_iters=k - 1)
    assert g_k <= eps * (1 + 1e-4)
    assert g_km1 > eps * (1 - 1e-4)


@pytest.mark.parametrize("C,H,W,K,prec", [(3, 70, 45, 7, adp.ADP_F32), (3, 256, 256, 15, adp.ADP_F32),
                                          (1, 64, 64, 7, adp.ADP_F64)])
def test_upper_loss(C, H, W, K, prec):
    pr = Pair(inst_for(C, H, W, K, kind="motion" if K >= 15 else "gauss"), prec=prec, beta=0.3)
    x = pr.rounded(pr.inst.x_true)
    b = pr.rounded(pr.inst.b_true)
    gx = torch.empty(pr.prob.img, dtype=pr.dt, device="cuda")
    loss, gxn = pr.prob.upper_loss(pr.t(b), pr.t(x), gradx=gx)
    lo, gno = pr.P.upper(pr.a, b, x, pr.y)
    _, go = pr.P.g(pr.a, x, pr.y)
    tol = OP_TOL[prec] * 2
    assert loss == pytest.approx(lo, rel=tol)
    assert gxn == pytest.approx(gno, rel=tol)
    # grad g = 2 A^T (A x - y) inherits the cancellation of the data residual:
    # each residual value carries an absolute error of about u * |A x| (u the
    # unit roundoff), i.e. a relative error of u * ||A x|| / ||A x - y||
    u = 2.0 ** -24 if prec == adp.ADP_F32 else 2.0 ** -53
    Ax = pr.P.conv(pr.a, x)
    kappa = np.linalg.norm(Ax) / np.linalg.norm(Ax - pr.y)
    assert rel(pr.n(gx), go) <= max(tol, 8 * u * kappa)


@pytest.mark.parametrize("C,H,W,K,prec", [(3, 70, 45, 7, adp.ADP_F32), (2, 33, 97, 15, adp.ADP_F32),
                                          (1, 64, 64, 7, adp.ADP_F64), (3, 256, 256, 15, adp.ADP_F32)])
def test_cross_term(C, H, W, K, prec):
    pr = Pair(inst_for(C, H, W, K), prec=prec)
    rng = np.random.default_rng(3)
    x = pr.rounded(pr.inst.x_true)
    v = pr.rounded(rng.standard_normal((C, H, W)))
    b = pr.rounded(pr.inst.b_true)
    out = pr.prob.cross_t(pr.t(b), pr.t(x), pr.t(v))
    assert rel(pr.n(out), pr.P.cross_t(b, x, pr.y, v)) <= (1e-6 if prec == adp.ADP_F32 else 1e-12)


@pytest.mark.parametrize("C,H,W,K,prec,n", [(3, 70, 45, 7, adp.ADP_F32, 12), (1, 64, 64, 7, adp.ADP_F64, 30),
                                            (3, 256, 256, 15, adp.ADP_F32, 3)])
def test_hypergrad_iteration_matched(C, H, W, K, prec, n):
    pr = Pair(inst_for(C, H, W, K, kind="motion" if K >= 15 else "gauss"), prec=prec, beta=0.3)
    b = pr.rounded(pr.inst.a)
    xg = pr.t(pr.rounded(pr.inst.y))
    pr.prob.lower_solve(pr.t(b), xg, eps=1e-2, max_iters=300)
    x = pr.n(xg)
    z, q, it, res, capped = pr.prob.hypergrad(pr.t(b), xg, delta=0.0, max_iters=n)
    zo, qo, ito, reso, cappedo = pr.P.hypergrad(pr.a, b, x, pr.y, delta=0.0, cg_max=n)
    assert it == ito == n
    tol = 1e-5 if prec == adp.ADP_F32 else 1e-11
    assert rel(pr.n(q), qo) <= tol
    assert rel(pr.n(z), zo) <= (1e-4 if prec == adp.ADP_F32 else 1e-10)
    assert res == pytest.approx(reso, rel=tol * 100)


def test_hypergrad_tolerance_matched_and_rhs():
    pr = Pair(inst_for(3, 70, 45, 7), prec=adp.ADP_F32, beta=0.3)
    b = pr.rounded(pr.inst.a)
    xg = pr.t(pr.rounded(pr.inst.y))
    pr.prob.lower_solve(pr.t(b), xg, eps=1e-3, max_iters=300)
    x = pr.n(xg)
    delta = 1e-3
    z, q, it, res, capped = pr.prob.hypergrad(pr.t(b), xg, delta=delta)
    zo, qo, ito, reso, _ = pr.P.hypergrad(pr.a, b, x, pr.y, delta=delta)
    assert not capped and res <= delta
    assert abs(it - ito) <= 1
    assert rel(pr.n(z), zo) <= 1e-4
    # explicit right-hand side (the autograd backward): no Sobolev term
    rhs = pr.rounded(np.random.default_rng(1).standard_normal(pr.prob.img))
    z2, q2, it2, _, _ = pr.prob.hypergrad(pr.t(b), xg, delta=1e-4, rhs=pr.t(rhs))
    zo2, _, ito2, _, _ = pr.P.hypergrad(pr.a, b, x, pr.y, delta=1e-4, rhs=rhs)
    assert abs(it2 - ito2) <= 1
    assert rel(pr.n(z2), zo2) <= 1e-4


def _maid_run(pr, steps, **over):
    """Run `steps` MAID iterations on both sides from the same state."""
    b0 = pr.rounded(pr.inst.a)
    x0 = pr.rounded(pr.inst.y)
    bg, xg = pr.t(b0), pr.t(x0)
    qg = torch.zeros_like(xg)
    sg = pr.prob.maid_init(**over)
    bo, xo = b0.copy(), x0.copy()
    so = pr.P.maid_init(pr.a, **over)
    log = []
    for _ in range(steps):
        acc_g = pr.prob.maid_step(sg, bg, xg, qg)
        acc_o, qo = pr.P.maid_step(so, pr.a, pr.y, bo, xo)
        log.append((acc_g, acc_o, sg.trials, so.trials, sg.rounds, so.rounds, sg.ll_iters, so.ll_iters,
                    sg.cg_iters, so.cg_iters, sg.psi, so.psi))
        assert acc_g == acc_o, log
        assert (sg.trials, sg.rounds) == (so.trials, so.rounds), log
        assert sg.eps == so.eps and sg.delta == so.delta and sg.step == so.step, log
    return (pr.n(bg), pr.n(xg), sg), (bo, xo, so), log


def test_maid_fp64_matches_oracle():
    inst = synth.make_instance("g", 1, 32, 32, synth.gaussian_kernel(7, 1.5), synth.gaussian_kernel(7, 1.0),
                               0.01, 0, texture=False)
    pr = Pair(inst, prec=adp.ADP_F64, beta=0.3)
    (bg, xg, sg), (bo, xo, so), log = _maid_run(pr, 3, eps=1e-4, delta=1e-4, step=1e-3)
    assert all(l[0] for l in log)
    assert rel(bg, bo) <= 1e-10 and rel(xg, xo) <= 1e-9
    assert sg.ll_iters == so.ll_iters and sg.cg_iters == so.cg_iters
    assert sg.loss == pytest.approx(so.loss, rel=1e-10)


def test_maid_fp32_matches_oracle_and_psnr():
    inst = synth.make_instance("m", 3, 64, 64, synth.motion_kernel(7, 5, 30), synth.motion_kernel(7, 5, 20),
                               0.02, 1)
    pr = Pair(inst, prec=adp.ADP_F32, beta=0.3)
    (bg, xg, sg), (bo, xo, so), log = _maid_run(pr, 3, eps=1e-3, delta=1e-3, step=1e-2)
    assert rel(bg, bo) <= 1e-4
    assert rel(xg, xo) <= 1e-4
    assert abs(psnr(xg, inst.x_true) - psnr(xo, inst.x_true)) <= 0.05
    kpeak = float(np.max(inst.b_true))
    assert abs(psnr(bg, inst.b_true, kpeak) - psnr(bo, inst.b_true, kpeak)) <= 0.05


def test_maid_line_search_exhaustion_reports_lsfail():
    inst = inst_for(1, 32, 32, 5)
    pr = Pair(inst, prec=adp.ADP_F64, beta=0.3)
    b, x = pr.t(pr.rounded(inst.a)), pr.t(pr.rounded(inst.y))
    b_before = b.clone()
    s = pr.prob.maid_init(step=1e12, max_rounds=1, max_bt=2)
    assert pr.prob.maid_step(s, b, x, torch.zeros_like(x)) is False
    assert torch.equal(b, b_before)
    assert s.eps == pytest.approx(5e-3) and s.step == pytest.approx(0.25e12) and s.trials == 2


def test_nonfinite_input_is_reported():
    inst = inst_for(1, 32, 32, 5)
    pr = Pair(inst, prec=adp.ADP_F32)
    x = pr.t(pr.rounded(inst.y))
    x[0, 3, 4] = float("nan")
    with pytest.raises(adp.AdpError) as e:
        pr.prob.lower_solve(pr.t(pr.rounded(inst.a)), x, eps=1e-3)
    assert e.value.status == adp.ADP_ENONFINITE
    # the context stays usable
    x2 = pr.t(pr.rounded(inst.y))
    pr.prob.lower_solve(pr.t(pr.rounded(inst.a)), x2, eps=1e-1)


def test_invalid_arguments_are_rejected():
    inst = inst_for(1, 16, 16, 3)
    y = torch.tensor(inst.y, dtype=torch.float32, device="cuda")
    a = torch.tensor(inst.a, dtype=torch.float32, device="cuda")
    with pytest.raises(adp.AdpError) as e:
        adp.Problem(adp.Params(1, 16, 16, 4), y, a.new_zeros((1, 4, 4)))
    assert e.value.status == adp.ADP_EINVAL
    with pytest.raises(adp.AdpError):
        adp.Problem(adp.Params(1, 16, 16, 65), y, a.new_zeros((1, 65, 65)))
    pr = adp.Problem(adp.Params(1, 16, 16, 3), y, a)
    with pytest.raises(TypeError):
        pr.apply_B(a.double(), y)


def test_problems_with_different_kernel_sizes_coexist():
    # the kernel's shared-memory opt-in is shared by all problems on a device:
    # creating a problem with a small K after one with a large K must not break
    # the large one's launches
    big = Pair(inst_for(1, 40, 40, 31), prec=adp.ADP_F32)
    small = Pair(inst_for(1, 40, 40, 3), prec=adp.ADP_F32)
    rng = np.random.default_rng(0)
    for pr in (big, small, big):
        x = pr.rounded(rng.uniform(size=(1, 40, 40)))
        b = pr.rounded(pr.inst.b_true)
        out = pr.prob.apply_B(pr.t(b), pr.t(x))
        assert rel(pr.n(out), pr.P.conv(b, x)) <= OP_TOL[adp.ADP_F32]


def test_maid_stop_rule_matches_oracle():
    inst = inst_for(1, 32, 32, 5)
    pr = Pair(inst, prec=adp.ADP_F64, beta=0.3)
    b, x = pr.t(pr.rounded(inst.a)), pr.t(pr.rounded(inst.y))
    s = pr.prob.maid_init(step=1e12, max_rounds=10, max_bt=2, eps_stop=3e-3)
    assert pr.prob.maid_step(s, b, x, torch.zeros_like(x)) is False
    so = pr.P.maid_init(pr.a, step=1e12, max_rounds=10, max_bt=2, eps_stop=3e-3)
    bo, xo = pr.rounded(inst.a), pr.rounded(inst.y)
    pr.P.maid_step(so, pr.a, pr.y, bo, xo)
    assert s.stopped == so.stopped == 1
    assert (s.rounds, s.trials, s.eps, s.step) == (so.rounds, so.trials, so.eps, so.step)
    # at entry: nothing runs
    s2 = pr.prob.maid_init(eps=1e-3, delta=1e-3, eps_stop=1e-3)
    assert pr.prob.maid_step(s2, b, x, torch.zeros_like(x)) is False
    assert s2.stopped == 1 and s2.ll_iters == 0 and s2.rounds == 0


def test_paper_2d_setting_fp64():
    """The paper's own 2D setting (Sec. 4.2) on a synthetic 300 x 400 RGB image:
    5 x 5 diagonal motion blur, sqrt-smoothed TV with nu = 1e-4, alpha 0.6,
    beta 0.3 on the H^1 seminorm, in FP64.  FISTA and CG iteration-matched
    against the oracle.  phi'' reaches 1/nu = 1e4 here, so the Hessian is far
    worse conditioned than in the other cases; the CG iterate and z are held
    to 1e-7 and 1e-6 (rounding-order differences amplified by that condition),
    the FISTA iterate to 1e-10."""
    inst = synth.paper2d_motion(0)
    pr = Pair(inst, prec=adp.ADP_F64, alpha=0.6, reg=adp.ADP_REG_SQRT_TV, reg_param=1e-4, beta=0.3, w0=0.0)
    x0, b = pr.rounded(inst.y), pr.rounded(inst.a)
    xg = pr.t(x0)
    it, gn, capped = pr.prob.lower_solve(pr.t(b), xg, eps=0.0, max_iters=20)
    xo, ito, gno = pr.P.fista(b, pr.y, x0, eps=0.0, max_iters=20)
    assert it == ito == 20 and capped
    assert rel(pr.n(xg), xo) <= 1e-10
    assert gn == pytest.approx(gno, rel=1e-8)
    z, q, it2, res, _ = pr.prob.hypergrad(pr.t(b), xg, delta=0.0, max_iters=5)
    zo, qo, ito2, reso, _ = pr.P.hypergrad(pr.a, b, pr.n(xg), pr.y, delta=0.0, cg_max=5)
    assert it2 == ito2 == 5
    assert rel(pr.n(q), qo) <= 1e-7
    assert rel(pr.n(z), zo) <= 1e-6
    pr.prob.close()
