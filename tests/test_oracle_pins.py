"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

* library routines: scipy.ndimage convolve/correlate with periodic wrap, np.roll;
* the convolution theorem: Fourier closed forms of the lower-level minimiser, of
  the CG solution and of the upper loss for the quadratic regulariser
  J = 1/2 ||D x||^2 under periodic boundaries (Eq. 2.5 with that J);
* adjoint identities <B x, z> = <x, B^T z>, <D x, w> = <x, D^T w>;
* closed-form values of phi, J, r on simple inputs;
* central finite differences of values against gradients and of gradients
  against Hessian-vector products;
* the a-posteriori bound of Lemma 2 and the sufficient decrease of Lemma 1;
* the MAID constants printed in Sec. 4.1 / 4.2 (tests/golden/paper_constants.json).
"""
import json
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
from paper_2502_09758_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# --------------------------------------------------------------- Fourier tools
def symbol(k2d, H, W):
    """DFT of a centred K x K kernel placed periodically on an H x W grid."""
    K = k2d.shape[0]
    r = (K - 1) // 2
    pad = np.zeros((H, W))
    for p in range(K):
        for q in range(K):
            pad[(p - r) % H, (q - r) % W] += k2d[p, q]
    return np.fft.fft2(pad)


def dsym(H, W):
    """|D_h^|^2 + |D_v^|^2 for periodic forward differences."""
    wh = 2 - 2 * np.cos(2 * np.pi * np.arange(W) / W)
    wv = 2 - 2 * np.cos(2 * np.pi * np.arange(H) / H)
    return wv[:, None] + wh[None, :]


def quad_lower_closed(b, y, alpha):
    """argmin 1/2||Bx-y||^2 + alpha/2 ||Dx||^2 via the convolution theorem."""
    C, H, W = y.shape
    out = np.empty_like(y)
    for c in range(C):
        Bh = symbol(b[c], H, W)
        out[c] = np.real(np.fft.ifft2(np.conj(Bh) * np.fft.fft2(y[c]) /
                                      (np.abs(Bh) ** 2 + alpha * dsym(H, W))))
    return out


def quad_hess_solve(b, rhs, alpha):
    C, H, W = rhs.shape
    out = np.empty_like(rhs)
    for c in range(C):
        Bh = symbol(b[c], H, W)
        out[c] = np.real(np.fft.ifft2(np.fft.fft2(rhs[c]) / (np.abs(Bh) ** 2 + alpha * dsym(H, W))))
    return out


def quad_mu(b, alpha, H, W):
    return min(float(np.min(np.abs(symbol(b[c], H, W)) ** 2 + alpha * dsym(H, W)))
               for c in range(b.shape[0]))


def fft_conv(k, x):
    C, H, W = x.shape
    return np.stack([np.real(np.fft.ifft2(symbol(k[c], H, W) * np.fft.fft2(x[c]))) for c in range(C)])


def sobolev_closed(b, a, beta, w0):
    """beta (w0 ||d||^2 + ||d(:,1:)-d(:,:-1)||^2 + ||d(1:,:)-d(:-1,:)||^2)."""
    d = b - a
    return beta * (w0 * np.sum(d ** 2) + np.sum(np.diff(d, axis=2) ** 2) + np.sum(np.diff(d, axis=1) ** 2))


def ell_closed(b, a, y, alpha, beta, w0=1.0):
    """Exact upper loss of the quadratic-J problem: ||A x^(b) - y||^2 + r(b)."""
    xh = quad_lower_closed(b, y, alpha)
    e = fft_conv(a, xh) - y
    return float(np.sum(e ** 2)) + sobolev_closed(b, a, beta, w0)


# ------------------------------------------------------------------ constants
def test_paper_constants_match_defaults(orc):
    g = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    P = orc.Problem(1, 8, 8, 3)
    s = P.maid_init(np.ones((1, 3, 3)) / 9)
    assert s.eps == g["maid_eps0"]["value"]
    assert s.delta == g["maid_eps0"]["value"]          # delta = eps (Sec. 4.2)
    assert s.ll_max_iters == g["maid_ll_cap"]["value"]
    assert s.rho_up == g["maid_rho_up"]["value"]
    assert s.rho_down == g["maid_rho_down"]["value"]
    assert s.nu_up == g["maid_nu_up"]["value"]
    assert s.nu_down == g["maid_nu_down"]["value"]
    assert s.step == g["maid_step0"]["value"]


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("C,H,W,K", [(1, 8, 8, 3), (3, 9, 11, 5), (2, 16, 13, 7), (1, 7, 7, 7)])
def test_conv_matches_scipy_wrap(orc, C, H, W, K):
    rng = np.random.default_rng(H * W + K)
    P = orc.Problem(C, H, W, K)
    b = rng.standard_normal(P.ker_shape)
    x = rng.standard_normal(P.img_shape)
    out = P.conv(b, x)
    adj = P.conv_adj(b, x)
    for c in range(C):
        np.testing.assert_allclose(out[c], ndi.convolve(x[c], b[c], mode="wrap"), rtol=0, atol=1e-12)
        np.testing.assert_allclose(adj[c], ndi.correlate(x[c], b[c], mode="wrap"), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out, fft_conv(b, x), atol=1e-11)


def test_conv_kernel_larger_than_image(orc):
    # K > H wraps several times; the convolution theorem still holds exactly.
    rng = np.random.default_rng(5)
    P = orc.Problem(1, 4, 6, 7)
    b = rng.standard_normal(P.ker_shape)
    x = rng.standard_normal(P.img_shape)
    np.testing.assert_allclose(P.conv(b, x), fft_conv(b, x), atol=1e-11)


def test_conv_identity_kernel(orc):
    P = orc.Problem(2, 6, 5, 5)
    b = np.zeros(P.ker_shape)
    b[:, 2, 2] = 1.0
    x = np.random.default_rng(1).standard_normal(P.img_shape)
    np.testing.assert_array_equal(P.conv(b, x), x)
    np.testing.assert_array_equal(P.conv_adj(b, x), x)


@pytest.mark.parametrize("C,H,W,K", [(1, 8, 8, 3), (3, 10, 7, 5), (1, 5, 9, 9)])
def test_adjoint_identities(orc, C, H, W, K):
    rng = np.random.default_rng(3)
    P = orc.Problem(C, H, W, K)
    b = rng.standard_normal(P.ker_shape)
    x, z = rng.standard_normal(P.img_shape), rng.standard_normal(P.img_shape)
    lhs, rhs = np.vdot(P.conv(b, x), z), np.vdot(x, P.conv_adj(b, z))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10
    for f, fa in ((P.dh, P.dh_adj), (P.dv, P.dv_adj)):
        l, r = np.vdot(f(x), z), np.vdot(x, fa(z))
        assert abs(l - r) <= 1e-12
    np.testing.assert_array_equal(P.dh(x), np.roll(x, -1, axis=2) - x)
    np.testing.assert_array_equal(P.dv(x), np.roll(x, -1, axis=1) - x)


# ---------------------------------------------------------------- regulariser
def test_phi_closed_forms(orc):
    g = 0.01
    Ph = orc.Problem(1, 4, 4, 1, reg=orc.REG_HUBER, reg_param=g)
    assert Ph.phi(0.5 * g) == pytest.approx(0.125 * g, rel=1e-15)
    assert Ph.phi(3 * g) == pytest.approx(2.5 * g, rel=1e-15)
    assert Ph.phi(-3 * g) == pytest.approx(2.5 * g, rel=1e-15)
    assert Ph.dphi(g) == 1.0 and Ph.ddphi(g) == 1.0 / g      # tie in the quadratic branch
    assert Ph.ddphi(1.0001 * g) == 0.0
    nu = 1e-4
    Ps = orc.Problem(1, 4, 4, 1, reg=orc.REG_SQRT, reg_param=nu)
    assert Ps.phi(0.0) == 0.0
    assert Ps.phi(3e-4) == pytest.approx(np.sqrt(10) * 1e-4 - 1e-4, rel=1e-12)
    assert Ps.ddphi(0.0) == pytest.approx(1.0 / nu, rel=1e-12)
    for P in (Ph, Ps):
        for t in (-0.3, -2e-3, 4e-3, 0.02, 0.7, 3e-5):
            hstep = 1e-7 * max(abs(t), 1e-3)
            fd = (P.phi(t + hstep) - P.phi(t - hstep)) / (2 * hstep)
            assert P.dphi(t) == pytest.approx(fd, rel=1e-6, abs=1e-9)
            fd2 = (P.dphi(t + hstep) - P.dphi(t - hstep)) / (2 * hstep)
            assert P.ddphi(t) == pytest.approx(fd2, rel=1e-5, abs=1e-6)


def test_J_on_step_image(orc):
    # A vertical edge of height s at one column: each row has two jumps (the
    # edge and the periodic wrap), no vertical differences.
    H, W, s = 6, 8, 0.4
    x = np.zeros((1, H, W))
    x[0, :, 3:] = s
    for reg, par in ((orc.REG_HUBER, 0.01), (orc.REG_SQRT, 1e-4), (orc.REG_QUAD, 0.0)):
        P = orc.Problem(1, H, W, 1, reg=reg, reg_param=par)
        assert P.J(x) == pytest.approx(2 * H * P.phi(s), rel=1e-14)


@pytest.mark.parametrize("reg,par", [(oracle.REG_HUBER, 0.05), (oracle.REG_SQRT, 0.02), (oracle.REG_QUAD, 0.0)])
def test_gradJ_and_hessJ_finite_differences(orc, reg, par):
    rng = np.random.default_rng(11)
    P = orc.Problem(2, 6, 7, 1, reg=reg, reg_param=par)
    x = rng.uniform(size=P.img_shape)
    v = rng.standard_normal(P.img_shape)
    h = 1e-6
    fd = (P.J(x + h * v) - P.J(x - h * v)) / (2 * h)
    assert np.vdot(P.gradJ(x), v) == pytest.approx(fd, rel=1e-6)
    fdg = (P.gradJ(x + h * v) - P.gradJ(x - h * v)) / (2 * h)
    assert rel(P.hessJ_vec(x, v), fdg) < 1e-5


# ---------------------------------------------------------------- lower level
@pytest.mark.parametrize("reg,par", [(oracle.REG_HUBER, 0.05), (oracle.REG_SQRT, 0.02)])
def test_grad_h_and_hess_h_finite_differences(orc, reg, par):
    rng = np.random.default_rng(7)
    P = orc.Problem(2, 8, 9, 3, alpha=0.1, reg=reg, reg_param=par)
    b = rng.uniform(size=P.ker_shape)
    x, y = rng.uniform(size=P.img_shape), rng.uniform(size=P.img_shape)
    v = rng.standard_normal(P.img_shape)
    h = 1e-6
    fd = (P.h(b, x + h * v, y) - P.h(b, x - h * v, y)) / (2 * h)
    assert np.vdot(P.grad_h(b, x, y), v) == pytest.approx(fd, rel=1e-7)
    fdg = (P.grad_h(b, x + h * v, y) - P.grad_h(b, x - h * v, y)) / (2 * h)
    assert rel(P.hess_h_vec(b, x, v), fdg) < 1e-5


def test_h_value_closed_form(orc):
    # identity kernel and x = y leave only alpha J(y)
    P = orc.Problem(1, 6, 6, 3, alpha=0.3, reg=orc.REG_QUAD)
    b = np.zeros(P.ker_shape)
    b[0, 1, 1] = 1
    y = np.random.default_rng(2).uniform(size=P.img_shape)
    assert P.h(b, y, y) == pytest.approx(0.3 * 0.5 * (np.sum((np.roll(y, -1, 2) - y) ** 2) +
                                                      np.sum((np.roll(y, -1, 1) - y) ** 2)), rel=1e-14)


def test_lipschitz_bounds_true_spectrum(orc):
    inst = synth.small(C=2, H=12, W=12, K=5)
    P = orc.Problem(2, 12, 12, 5, alpha=0.2, reg=orc.REG_QUAD)
    for c in range(2):
        true = float(np.max(np.abs(symbol(inst.a[c], 12, 12)) ** 2 + 0.2 * dsym(12, 12)))
        L = P.lipschitz(inst.a, c)
        assert L >= true * (1 - 1e-12)
        # nonnegative normalised kernel: ||b||_1^2 = 1 = |B^(0)|^2, and max |D^|^2 = 8
        assert L == pytest.approx(1.0 + 8 * 0.2, rel=1e-12)


def test_fista_reaches_fourier_minimiser(orc):
    inst = synth.small(C=2, H=16, W=12, K=5, seed=4)
    alpha = 0.05
    P = orc.Problem(2, 16, 12, 5, alpha=alpha, reg=orc.REG_QUAD)
    xh = quad_lower_closed(inst.a, inst.y, alpha)
    x, it, gn = P.fista(inst.a, inst.y, inst.y, eps=1e-11, max_iters=100000)
    assert gn <= 1e-11 and it > 0
    assert rel(x, xh) < 1e-10


def test_fista_lemma2_aposteriori_bound(orc):
    inst = synth.small(C=1, H=16, W=16, K=3, seed=8)
    alpha = 0.02
    P = orc.Problem(1, 16, 16, 3, alpha=alpha, reg=orc.REG_QUAD)
    xh = quad_lower_closed(inst.a, inst.y, alpha)
    mu = quad_mu(inst.a, alpha, 16, 16)
    last = -1
    for eps in (1e-1, 1e-2, 1e-3, 1e-5):
        x, it, gn = P.fista(inst.a, inst.y, inst.y, eps=eps, max_iters=100000)
        assert gn <= eps
        assert it >= last            # tighter tolerance never needs fewer updates
        last = it
        assert np.linalg.norm(x - xh) <= gn / mu * (1 + 1e-9)
        # returned point satisfies the test it reports
        assert np.linalg.norm(P.grad_h(inst.a, x, inst.y)) == pytest.approx(gn, rel=1e-12)


def test_fista_warm_start_and_cap(orc):
    inst = synth.small(C=1, H=12, W=12, K=3, seed=9)
    P = orc.Problem(1, 12, 12, 3, alpha=0.01)
    x1, it1, gn1 = P.fista(inst.a, inst.y, inst.y, eps=1e-4, max_iters=10000)
    x2, it2, gn2 = P.fista(inst.a, inst.y, x1, eps=1e-4, max_iters=10000)
    assert it2 == 0 and gn2 == gn1 and np.array_equal(x1, x2)     # test passes at once
    x3, it3, gn3 = P.fista(inst.a, inst.y, inst.y, eps=1e-12, max_iters=7)
    assert it3 == 7 and gn3 > 1e-12


def test_cg_matches_fourier_solution(orc):
    inst = synth.small(C=2, H=10, W=14, K=3, seed=12)
    alpha = 0.1
    P = orc.Problem(2, 10, 14, 3, alpha=alpha, reg=orc.REG_QUAD)
    rhs = np.random.default_rng(0).standard_normal(P.img_shape)
    q, it, res, capped = P.cg(inst.a, inst.y, rhs, delta=1e-12, max_iters=5000)
    assert not capped and res <= 1e-12
    assert rel(q, quad_hess_solve(inst.a, rhs, alpha)) < 1e-10
    # warm start from the solution needs no iteration
    q2, it2, res2, _ = P.cg(inst.a, inst.y, rhs, delta=1e-10, q0=q)
    assert it2 == 0


def test_cg_huber_residual(orc):
    inst = synth.small(C=1, H=12, W=12, K=5, seed=13)
    P = orc.Problem(1, 12, 12, 5, alpha=0.01, reg_param=0.01)
    x, _, _ = P.fista(inst.a, inst.y, inst.y, eps=1e-8, max_iters=20000)
    rhs = P.g(inst.a, x, inst.y)[1]
    q, it, res, capped = P.cg(inst.a, x, rhs, delta=1e-9, max_iters=5000)
    assert not capped
    assert np.linalg.norm(P.hess_h_vec(inst.a, x, q) - rhs) <= 1e-9 * 1.001


# ---------------------------------------------------------------- upper level
def test_g_and_r_closed_forms(orc):
    rng = np.random.default_rng(21)
    P = orc.Problem(3, 9, 8, 5, beta=0.7, w0=1.0)
    a, b = rng.uniform(size=P.ker_shape), rng.uniform(size=P.ker_shape)
    x, y = rng.uniform(size=P.img_shape), rng.uniform(size=P.img_shape)
    val, grad = P.g(a, x, y)
    assert val == pytest.approx(float(np.sum((fft_conv(a, x) - y) ** 2)), rel=1e-12)
    v = rng.standard_normal(P.img_shape)
    h = 1e-6
    fd = (P.g(a, x + h * v, y)[0] - P.g(a, x - h * v, y)[0]) / (2 * h)
    assert np.vdot(grad, v) == pytest.approx(fd, rel=1e-7)
    rv, rg = P.r(b, a)
    assert rv == pytest.approx(sobolev_closed(b, a, 0.7, 1.0), rel=1e-13)
    w = rng.standard_normal(P.ker_shape)
    fd = (P.r(b + h * w, a)[0] - P.r(b - h * w, a)[0]) / (2 * h)
    assert np.vdot(rg, w) == pytest.approx(fd, rel=1e-7)
    # seminorm: adding a constant to b - a changes nothing
    P0 = orc.Problem(3, 9, 8, 5, beta=0.7, w0=0.0)
    assert P0.r(b + 0.25, a)[0] == pytest.approx(P0.r(b, a)[0], rel=1e-12)
    np.testing.assert_allclose(P0.r(b + 0.25, a)[1], P0.r(b, a)[1], atol=1e-13)
    # full norm of a constant deviation: only the w0 term survives
    assert P.r(a + 0.5, a)[0] == pytest.approx(0.7 * 3 * 25 * 0.25, rel=1e-14)
    assert P.L_gx(a) == pytest.approx(2 * max(np.sum(np.abs(a[c])) ** 2 for c in range(3)), rel=1e-14)
    lu, gn = P.upper(a, b, x, y)
    assert lu == pytest.approx(val + rv, rel=1e-14) and gn == pytest.approx(np.linalg.norm(grad), rel=1e-13)


def test_hypergradient_matches_closed_form_finite_differences(orc):
    # quadratic J: ell(b) = ||A x^(b) - y||^2 + r(b) has an FFT closed form, so
    # the IFT hypergradient (FISTA + CG + cross term) can be checked against
    # central differences that never touch the oracle.
    inst = synth.small(C=2, H=10, W=12, K=3, seed=31)
    alpha, beta = 0.05, 0.3
    P = orc.Problem(2, 10, 12, 3, alpha=alpha, reg=orc.REG_QUAD, beta=beta)
    b = inst.a + 0.03 * np.random.default_rng(1).standard_normal(inst.a.shape)
    x, _, _ = P.fista(b, inst.y, inst.y, eps=1e-13, max_iters=200000)
    z, q, it, res, capped = P.hypergrad(inst.a, b, x, inst.y, delta=1e-13, cg_max=20000)
    assert not capped
    h = 1e-6
    fd = np.zeros_like(b)
    for idx in np.ndindex(*b.shape):
        bp, bm = b.copy(), b.copy()
        bp[idx] += h
        bm[idx] -= h
        fd[idx] = (ell_closed(bp, inst.a, inst.y, alpha, beta) - ell_closed(bm, inst.a, inst.y, alpha, beta)) / (2 * h)
    assert rel(z, fd) < 1e-6


def test_hypergradient_huber_finite_differences(orc):
    # Smoothed-TV lower level: compare the IFT hypergradient with differences of
    # ell(b) = g(x~(b)) + r(b) from tightly solved lower problems.
    inst = synth.small(C=1, H=8, W=8, K=3, seed=41, noise=0.02)
    alpha, beta = 0.02, 0.3
    P = orc.Problem(1, 8, 8, 3, alpha=alpha, reg=orc.REG_SQRT, reg_param=0.05, beta=beta)
    b = inst.a.copy()
    x, _, gn = P.fista(b, inst.y, inst.y, eps=1e-12, max_iters=400000)
    assert gn <= 1e-12
    z, q, it, res, capped = P.hypergrad(inst.a, b, x, inst.y, delta=1e-12, cg_max=20000)
    assert not capped

    def ell(bb):
        xx, _, g2 = P.fista(bb, inst.y, x, eps=1e-12, max_iters=400000)
        assert g2 <= 1e-12
        return P.upper(inst.a, bb, xx, inst.y)[0]

    h = 1e-5
    fd = np.zeros_like(b)
    for idx in np.ndindex(*b.shape):
        bp, bm = b.copy(), b.copy()
        bp[idx] += h
        bm[idx] -= h
        fd[idx] = (ell(bp) - ell(bm)) / (2 * h)
    assert rel(z, fd) < 1e-5


def test_hypergradient_rhs_variant(orc):
    # with an explicit right-hand side the Sobolev term is left out and the
    # result is linear in the right-hand side
    inst = synth.small(C=1, H=8, W=10, K=3, seed=51)
    P = orc.Problem(1, 8, 10, 3, alpha=0.05, reg=orc.REG_QUAD, beta=0.3)
    rng = np.random.default_rng(0)
    x = inst.y
    r1, r2 = rng.standard_normal(P.img_shape), rng.standard_normal(P.img_shape)
    z1 = P.hypergrad(inst.a, inst.a, x, inst.y, 1e-13, rhs=r1, cg_max=5000)[0]
    z2 = P.hypergrad(inst.a, inst.a, x, inst.y, 1e-13, rhs=r2, cg_max=5000)[0]
    z12 = P.hypergrad(inst.a, inst.a, x, inst.y, 1e-13, rhs=r1 + 2 * r2, cg_max=5000)[0]
    assert rel(z12, z1 + 2 * z2) < 1e-9
    g = P.g(inst.a, x, inst.y)[1]
    zg = P.hypergrad(inst.a, inst.a, x, inst.y, 1e-13, rhs=g, cg_max=5000)[0]
    zf = P.hypergrad(inst.a, inst.a, x, inst.y, 1e-13, cg_max=5000)[0]
    assert rel(zf - zg, P.r(inst.a, inst.a)[1]) < 1e-9 or np.allclose(zf, zg)


# ---------------------------------------------------------------------- MAID
def test_maid_lemma1_sufficient_decrease(orc):
    # Accepted MAID steps must decrease the exact upper loss (closed form) by at
    # least lambda * step * ||z||^2 (Lemma 1).
    inst = synth.small(C=1, H=12, W=12, K=3, seed=61, noise=0.02, sigma_true=1.0, sigma_init=0.6)
    alpha, beta = 0.05, 0.1
    P = orc.Problem(1, 12, 12, 3, alpha=alpha, reg=orc.REG_QUAD, beta=beta)
    # the paper's eps0 = 1e-2 is sized for 300 x 400 x 3 images; on 12 x 12 the
    # error terms of psi need a tighter start
    s = P.maid_init(inst.a, ll_max_iters=100000, cg_max_iters=20000, eps=1e-6, delta=1e-6, step=1e-3)
    b, x = inst.a.copy(), inst.y.copy()
    accepted = 0
    for _ in range(8):
        step, eps = s.step, s.eps
        l_before = ell_closed(b, inst.a, inst.y, alpha, beta)
        acc, q = P.maid_step(s, inst.a, inst.y, b, x)
        assert acc
        accepted += 1
        l_after = ell_closed(b, inst.a, inst.y, alpha, beta)
        used_step = s.step / s.rho_up
        assert l_after - l_before <= -s.lam * used_step * s.znorm ** 2 + 1e-14
        # Algorithm 2 updates: eps and delta grow by nu_up after success
        assert s.eps == pytest.approx(s.delta)
        assert used_step <= step * (1 + 1e-15)
    assert accepted == 8 and s.k == 8


def test_maid_large_beta_keeps_kernel(orc):
    inst = synth.small(C=1, H=10, W=10, K=3, seed=71)
    P = orc.Problem(1, 10, 10, 3, alpha=0.05, reg=orc.REG_HUBER, reg_param=0.01, beta=1e4)
    s = P.maid_init(inst.a, step=1e-6)
    b, x = inst.a.copy(), inst.y.copy()
    for _ in range(3):
        P.maid_step(s, inst.a, inst.y, b, x)
    assert np.max(np.abs(b - inst.a)) < 1e-4


def test_maid_backtracking_exhaustion(orc):
    # a tiny number of rounds with an absurd first step: the line search fails,
    # b is unchanged and eps, delta and the step have all shrunk
    inst = synth.small(C=1, H=8, W=8, K=3, seed=81)
    P = orc.Problem(1, 8, 8, 3, alpha=0.05, reg=orc.REG_QUAD, beta=0.3)
    s = P.maid_init(inst.a, step=1e12, max_rounds=1, max_bt=2)
    b, x = inst.a.copy(), inst.y.copy()
    acc, _ = P.maid_step(s, inst.a, inst.y, b, x)
    assert not acc
    np.testing.assert_array_equal(b, inst.a)
    assert s.eps == pytest.approx(0.5e-2) and s.delta == pytest.approx(0.5e-2)
    assert s.step == pytest.approx(1e12 * 0.25) and s.trials == 2


def test_maid_stop_rule_sec42(orc):
    # Sec. 4.2: the upper iterations end when MAID's accuracy reaches the stop
    # tolerance.  At entry: no work at all.  During backtracking: the step ends
    # as soon as a failed round has shrunk eps to the tolerance.
    inst = synth.small(C=1, H=8, W=8, K=3, seed=82)
    P = orc.Problem(1, 8, 8, 3, alpha=0.05, reg=orc.REG_QUAD, beta=0.3)
    s = P.maid_init(inst.a, eps=1e-3, delta=1e-3, eps_stop=1e-3)
    b, x = inst.a.copy(), inst.y.copy()
    acc, _ = P.maid_step(s, inst.a, inst.y, b, x)
    assert not acc and s.stopped == 1 and s.ll_iters == 0 and s.rounds == 0
    np.testing.assert_array_equal(x, inst.y)
    s = P.maid_init(inst.a, step=1e12, max_rounds=10, max_bt=2, eps_stop=3e-3)
    acc, _ = P.maid_step(s, inst.a, inst.y, b, x)
    assert not acc and s.stopped == 1 and s.rounds == 2          # 1e-2 -> 5e-3 -> 2.5e-3
    assert s.eps == pytest.approx(2.5e-3) and s.trials == 2 + 3
    np.testing.assert_array_equal(b, inst.a)


# ------------------------------------------------------------ single outputs
@pytest.mark.parametrize("reg,par", [(oracle.REG_HUBER, 0.05), (oracle.REG_SQRT, 0.1), (oracle.REG_QUAD, 1.0)])
def test_single_output_functions_match_whole_image(orc, reg, par):
    """The per-pixel evaluations used for sampled checks at large sizes agree
    with the whole-image functions (themselves pinned above) at every pixel,
    including the periodic wrap at all four edges and a kernel wider than the
    image."""
    for C, H, W, K in [(2, 9, 11, 5), (1, 6, 5, 7)]:
        rng = np.random.default_rng(C * 100 + K)
        P = oracle.Problem(C, H, W, K, alpha=0.3, reg=reg, reg_param=par)
        b = rng.standard_normal((C, K, K))
        x, y, v = (rng.standard_normal((C, H, W)) for _ in range(3))
        idx = [(c, i, j) for c in range(C) for i in range(H) for j in range(W)]
        np.testing.assert_allclose(P.conv_at(b, x, idx), P.conv(b, x).ravel(), rtol=0, atol=1e-13)
        np.testing.assert_allclose(P.conv_adj_at(b, x, idx), P.conv_adj(b, x).ravel(), rtol=0, atol=1e-13)
        np.testing.assert_allclose(P.grad_h_at(b, x, y, idx), P.grad_h(b, x, y).ravel(), rtol=0, atol=1e-11)
        np.testing.assert_allclose(P.hess_h_vec_at(b, x, v, idx), P.hess_h_vec(b, x, v).ravel(), rtol=0,
                                   atol=1e-11)


# ------------------------------------------------------------ BF16 operands
def test_bf16_round_definition():
    """Round to nearest, ties to even, at 8 significant bits (spacing 2^-7 on
    [1, 2)): representable values stay, midpoints go to the even neighbour,
    anything past a midpoint goes up; the input is first rounded to FP32."""
    r = oracle.bf16_round
    exact = np.array([0.0, 1.0, -3.5, 1 + 2.0 ** -7, 2.0 ** -126, 1.5 * 2.0 ** 100, -(1 + 127 * 2.0 ** -7)])
    np.testing.assert_array_equal(r(exact), exact)
    assert r(1 + 2.0 ** -8) == 1.0                          # tie, 1 is even
    assert r(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6            # tie, 1 + 2^-6 is even
    assert r(-(1 + 2.0 ** -8)) == -1.0
    assert r(1 + 2.0 ** -8 + 2.0 ** -20) == 1 + 2.0 ** -7   # past the tie
    assert r(1 + 2.0 ** -8 - 2.0 ** -20) == 1.0
    assert r(1 + 2.0 ** -8 + 2.0 ** -30) == 1.0             # FP32 first: the 2^-30 is gone
    assert r(2 - 2.0 ** -9) == 2.0                          # carry into the exponent
    rng = np.random.default_rng(3)
    v = rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))
    q = r(v)
    v32 = v.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(q - v32) <= 2.0 ** -8 * np.abs(v32))   # unit roundoff of 8 significant bits
    assert np.all(np.diff(q[np.argsort(v32)]) >= 0)             # monotone
    # the low 16 bits of every result are zero
    assert np.all(q.astype(np.float32).view(np.uint32) & 0xFFFF == 0)


def test_bf16_round_matches_torch_conversion():
    """Special case that reduces to a library routine: PyTorch's CPU
    float32 -> bfloat16 conversion also rounds to nearest even."""
    import torch
    rng = np.random.default_rng(4)
    v = (rng.standard_normal(50000) * np.exp(rng.uniform(-30, 30, 50000))).astype(np.float32)
    t = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.bf16_round(v), t)

