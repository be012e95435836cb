"""Pins of the oracle's iterates, not only of its fixed points.

The GPU parity tests compare the n-th iterate of FISTA and CG and the accept /
reject decisions of MAID with the oracle, so the oracle's trajectory itself
must be right.  Each pin below computes the expected value by a route that
shares nothing with the oracle's spatial loops:

* FISTA (Algorithm 1, step 1; the accelerated solver of Sec. 4.2): with the
  quadratic regulariser J = 1/2 ||D x||^2 and periodic boundaries the Hessian
  of h is diagonal in the Fourier basis, so every Fourier mode follows the
  scalar FISTA recurrence x_{k+1} = y_k - tau (lam_w y_k - c_w),
  y_{k+1} = x_{k+1} + theta_k (x_{k+1} - x_k), with t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
  and theta_k = (t_k - 1) / t_{k+1} (Beck and Teboulle's momentum), and
  tau = 1 / (||b_c||_1^2 + 8 alpha) per channel.  The n-th iterate follows from
  NumPy's FFT mode by mode.
* CG (Algorithm 1, step 2): the n-th CG iterate is the minimiser of the
  H-norm error over q_0 + span{r_0, H r_0, ..., H^{n-1} r_0}; the test builds
  that Krylov space explicitly from a dense H, orthonormalises it and solves
  the n x n Galerkin system.
* psi (Eq. 3.4): every term of the reported psi is recomputed from the
  problem's closed forms (FFT convolution for g and grad g, the Sobolev norm
  written with np.diff), and the exact decrease of Lemma 1 is checked at loose
  accuracies on problems whose strong-convexity constant is at least 1, so
  that ||grad_x h|| <= eps bounds ||x~ - x^|| by eps as Eq. 3.4 assumes.
"""
import numpy as np
import pytest

import oracle
from paper_2502_09758_gb300 import synth

from test_oracle_pins import dsym, fft_conv, quad_lower_closed, quad_mu, rel, sobolev_closed, symbol


# ------------------------------------------------------------------ FISTA
def fista_fourier(b, y, x0, alpha, n):
    """n FISTA updates of 1/2||Bx - y||^2 + alpha/2 ||Dx||^2 from x0, mode by
    mode in the Fourier domain; returns y_n (the point the solver returns)."""
    C, H, W = y.shape
    out = np.empty_like(y)
    for c in range(C):
        Bh = symbol(b[c], H, W)
        lam = np.abs(Bh) ** 2 + alpha * dsym(H, W)
        chat = np.conj(Bh) * np.fft.fft2(y[c])
        tau = 1.0 / (np.sum(np.abs(b[c])) ** 2 + 8.0 * alpha)
        X = np.fft.fft2(x0[c])
        Y = X.copy()
        t = 1.0
        for _ in range(n):
            Xn = Y - tau * (lam * Y - chat)
            tn = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            Y = Xn + ((t - 1.0) / tn) * (Xn - X)
            X, t = Xn, tn
        out[c] = np.real(np.fft.ifft2(Y))
    return out


def signed_kernels(C, K, seed):
    """Kernels with mixed signs and sums != 1, so that ||b_c||_1 differs from
    |sum b_c| and the step differs between channels."""
    rng = np.random.default_rng(seed)
    g = synth.gaussian_kernel(K, 1.0)
    return np.stack([(1.0 + 0.4 * c) * g + 0.05 * rng.standard_normal((K, K)) for c in range(C)])


@pytest.mark.parametrize("n", [1, 2, 5, 20])
def test_fista_nth_iterate_fourier_recurrence(orc, n):
    C, H, W, K, alpha = 2, 16, 12, 5, 0.07
    b = signed_kernels(C, K, 3)
    rng = np.random.default_rng(100 + n)
    y = rng.uniform(size=(C, H, W))
    x0 = rng.uniform(size=(C, H, W))
    P = orc.Problem(C, H, W, K, alpha=alpha, reg=orc.REG_QUAD)
    xn, it, _ = P.fista(b, y, x0, eps=0.0, max_iters=n)
    assert it == n
    ref = fista_fourier(b, y, x0, alpha, n)
    assert rel(xn, ref) < 1e-12
    # the iterate moves: a plain gradient step (theta = 0) differs from it
    if n >= 2:
        assert rel(ref, fista_fourier_no_momentum(b, y, x0, alpha, n)) > 1e-6


def fista_fourier_no_momentum(b, y, x0, alpha, n):
    C, H, W = y.shape
    out = np.empty_like(y)
    for c in range(C):
        Bh = symbol(b[c], H, W)
        lam = np.abs(Bh) ** 2 + alpha * dsym(H, W)
        chat = np.conj(Bh) * np.fft.fft2(y[c])
        tau = 1.0 / (np.sum(np.abs(b[c])) ** 2 + 8.0 * alpha)
        Y = np.fft.fft2(x0[c])
        for _ in range(n):
            Y = Y - tau * (lam * Y - chat)
        out[c] = np.real(np.fft.ifft2(Y))
    return out


def test_fista_stops_at_first_passing_iterate(orc):
    """The solver returns y_k for the first k whose gradient norm passes the
    test; the gradient norm of each Fourier-recurrence iterate, evaluated with
    the closed-form spectrum, decides which k that is."""
    C, H, W, K, alpha = 1, 16, 16, 3, 0.05
    inst = synth.small(C=C, H=H, W=W, K=K, seed=5)
    P = orc.Problem(C, H, W, K, alpha=alpha, reg=orc.REG_QUAD)
    Bh = symbol(inst.a[0], H, W)
    lam = np.abs(Bh) ** 2 + alpha * dsym(H, W)

    def gradnorm(v):
        G = lam * np.fft.fft2(v[0]) - np.conj(Bh) * np.fft.fft2(inst.y[0])
        return float(np.linalg.norm(np.fft.ifft2(G).real))

    norms = [gradnorm(fista_fourier(inst.a, inst.y, inst.y, alpha, k)) for k in range(60)]
    eps = 0.5 * (norms[20] + norms[21])
    k_first = next(k for k, g in enumerate(norms) if g <= eps)
    x, it, gn = P.fista(inst.a, inst.y, inst.y, eps=eps, max_iters=1000)
    assert it == k_first
    assert gn == pytest.approx(norms[k_first], rel=1e-10)
    assert rel(x, fista_fourier(inst.a, inst.y, inst.y, alpha, k_first)) < 1e-12


# --------------------------------------------------------------------- CG
def dense_hessian(P, b, x):
    n = int(np.prod(P.img_shape))
    Hm = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        Hm[:, k] = P.hess_h_vec(b, x, e.reshape(P.img_shape)).ravel()
    return 0.5 * (Hm + Hm.T)


def krylov_iterate(Hm, rhs, q0, n):
    """argmin over q0 + K_n(H, r0) of the H-norm error: orthonormal basis of
    the Krylov space, then the Galerkin system V^T H V c = V^T r0."""
    r0 = rhs - Hm @ q0
    cols = [r0 / np.linalg.norm(r0)]
    for _ in range(n - 1):
        v = Hm @ cols[-1]
        for u in cols:                       # two passes of Gram-Schmidt
            v -= (u @ v) * u
        for u in cols:
            v -= (u @ v) * u
        cols.append(v / np.linalg.norm(v))
    V = np.stack(cols, axis=1)
    c = np.linalg.solve(V.T @ Hm @ V, V.T @ r0)
    return q0 + V @ c


@pytest.mark.parametrize("reg,par", [(oracle.REG_QUAD, 0.0), (oracle.REG_HUBER, 0.05)])
def test_cg_nth_iterate_is_krylov_minimiser(orc, reg, par):
    C, H, W, K = 1, 8, 8, 3
    inst = synth.small(C=C, H=H, W=W, K=K, seed=17)
    P = orc.Problem(C, H, W, K, alpha=0.05, reg=reg, reg_param=par)
    rng = np.random.default_rng(7)
    x = rng.uniform(size=P.img_shape) * 0.2          # Huber: a mix of both branches of phi''
    rhs = rng.standard_normal(P.img_shape)
    q0 = 0.3 * rng.standard_normal(P.img_shape)
    Hm = dense_hessian(P, inst.a, x)
    assert np.min(np.linalg.eigvalsh(Hm)) > 0
    qstar = np.linalg.solve(Hm, rhs.ravel())
    prev = np.inf
    for n in (1, 2, 3, 4, 6):
        q, it, _, _ = P.cg(inst.a, x, rhs, delta=0.0, max_iters=n, q0=q0)
        assert it == n
        ref = krylov_iterate(Hm, rhs.ravel(), q0.ravel(), n)
        assert rel(q.ravel(), ref) < 1e-9, n
        e = q.ravel() - qstar
        err = float(e @ Hm @ e)
        assert err <= prev * (1 + 1e-12)             # the H-norm error never grows
        prev = err
    # a steepest-descent step is not the Krylov minimiser at n = 2
    r0 = rhs.ravel() - Hm @ q0.ravel()
    sd = q0.ravel().copy()
    r = r0.copy()
    for _ in range(2):
        a = (r @ r) / (r @ Hm @ r)
        sd += a * r
        r -= a * (Hm @ r)
    assert rel(sd, krylov_iterate(Hm, rhs.ravel(), q0.ravel(), 2)) > 1e-6


# -------------------------------------------------------------------- psi
def closed_upper(a, b, x, y, beta, w0):
    """ell = ||A x - y||^2 + r(b) and ||grad g|| = ||2 A^T (A x - y)|| through
    the convolution theorem and np.diff (no oracle call)."""
    C, H, W = x.shape
    e = fft_conv(a, x) - y
    gg = np.stack([2.0 * np.real(np.fft.ifft2(np.conj(symbol(a[c], H, W)) * np.fft.fft2(e[c])))
                   for c in range(C)])
    return float(np.sum(e ** 2)) + sobolev_closed(b, a, beta, w0), float(np.linalg.norm(gg))


def psi_closed(l0, gx0, l1, gx1, eps, L, lam, step, zz):
    """Eq. 3.4 with eps_bar = eps_k."""
    return l1 + gx1 * eps + 0.5 * L * eps * eps - l0 + gx0 * eps + lam * step * zz


def l_gx_closed(a):
    return 2.0 * max(float(np.sum(np.abs(a[c]))) ** 2 for c in range(a.shape[0]))


def psi_case(orc, seed, eps, step, reg):
    inst = synth.small(C=1, H=12, W=12, K=3, seed=seed, noise=0.02, sigma_true=1.0, sigma_init=0.6)
    alpha, beta = 0.05, 0.1
    P = orc.Problem(1, 12, 12, 3, alpha=alpha, reg=reg, reg_param=0.05, beta=beta)
    return inst, P, alpha, beta


@pytest.mark.parametrize("seed,eps,step,reg", [
    (61, 1e-3, 1e-2, oracle.REG_QUAD), (61, 3e-4, 1e-3, oracle.REG_QUAD),
    (61, 3e-4, 3e-4, oracle.REG_HUBER), (62, 1e-4, 3e-3, oracle.REG_QUAD),
    (62, 1e-4, 1e-3, oracle.REG_HUBER)])
def test_psi_reported_value_has_eq34_decomposition_accepted(orc, seed, eps, step, reg):
    """An accepted first trial: x~(b_k) is the oracle's warm-started solve, z is
    read back from b_{k+1} = b_k - alpha z, and each term of psi is recomputed
    from the closed forms."""
    inst, P, alpha, beta = psi_case(orc, seed, eps, step, reg)
    s = P.maid_init(inst.a, eps=eps, delta=eps, step=step, max_rounds=1, max_bt=1)
    b, x = inst.a.copy(), inst.y.copy()
    xk, _, _ = P.fista(b, inst.y, x, eps=eps)          # x~(b_k), as the step computes it
    acc, _ = P.maid_step(s, inst.a, inst.y, b, x)
    assert acc and s.rounds == 1 and s.trials == 1
    z = (inst.a - b) / step
    l0, gx0 = closed_upper(inst.a, inst.a, xk, inst.y, beta, 1.0)
    l1, gx1 = closed_upper(inst.a, b, x, inst.y, beta, 1.0)
    zz = float(np.sum(z ** 2))
    ref = psi_closed(l0, gx0, l1, gx1, eps, l_gx_closed(inst.a), s.lam, step, zz)
    scale = abs(l0) + abs(l1) + (gx0 + gx1) * eps
    assert abs(s.psi - ref) <= 1e-11 * scale
    assert ref <= 0.0
    assert s.znorm == pytest.approx(np.sqrt(zz), rel=1e-9)
    assert s.loss == pytest.approx(l1, rel=1e-12) and s.gradx_norm == pytest.approx(gx1, rel=1e-10)
    # each term is resolved by the tolerance above
    for term in ((gx0 + gx1) * eps, 0.5 * l_gx_closed(inst.a) * eps * eps, s.lam * step * zz):
        assert term > 1e3 * 1e-11 * scale


@pytest.mark.parametrize("seed,eps,step", [(71, 1e-2, 10.0), (72, 3e-3, 3.0)])
def test_psi_reported_value_has_eq34_decomposition_rejected(orc, seed, eps, step):
    """A rejected line search: psi of the last trial (step alpha_0 rho_down^(j-1))
    against the closed form at that step, and psi > 0 for every trial."""
    inst, P, alpha, beta = psi_case(orc, seed, eps, step, oracle.REG_QUAD)
    s = P.maid_init(inst.a, eps=eps, delta=eps, step=step, max_rounds=1, max_bt=3)
    b, x = inst.a.copy(), inst.y.copy()
    xk, _, _ = P.fista(b, inst.y, x, eps=eps)
    z, _, _, _, _ = P.hypergrad(inst.a, b, xk, inst.y, eps)
    acc, _ = P.maid_step(s, inst.a, inst.y, b, x)
    assert not acc and s.trials == 3
    np.testing.assert_array_equal(b, inst.a)
    l0, gx0 = closed_upper(inst.a, inst.a, xk, inst.y, beta, 1.0)
    zz = float(np.sum(z ** 2))
    for i in range(3):
        st = step * 0.5 ** i
        bt = inst.a - st * z
        xt, _, _ = P.fista(bt, inst.y, xk, eps=eps)
        l1, gx1 = closed_upper(inst.a, bt, xt, inst.y, beta, 1.0)
        ref = psi_closed(l0, gx0, l1, gx1, eps, l_gx_closed(inst.a), s.lam, st, zz)
        assert ref > 0.0
    scale = abs(l0) + abs(l1) + (gx0 + gx1) * eps
    assert abs(s.psi - ref) <= 1e-11 * scale
    assert s.step == pytest.approx(step * 0.5 ** 3)


def strongly_convex_instance(seed):
    """Semi-blind 3 x 3 problem whose kernels all have |B^(w)| >= 1.26 at every
    frequency (a mild five-point blur with sum 1.5), so that
    mu = min_w |B^|^2 + alpha |D^|^2 >= 1 along the whole run."""
    rng = np.random.default_rng(seed)
    x = synth.piecewise_image(rng, 1, 12, 12)

    def k(s):
        return 1.5 * np.array([[0.0, s, 0.0], [s, 1.0 - 4.0 * s, s], [0.0, s, 0.0]])

    y = fft_conv(k(0.1)[None], x) + 0.02 * rng.standard_normal(x.shape)
    return k(0.02)[None].copy(), y


@pytest.mark.parametrize("seed", [81, 82, 83, 84])
def test_lemma1_exact_decrease_over_steps_and_accuracies(orc, seed):
    """Lemma 1: a trial accepted by psi <= 0 decreases the exact upper loss
    (closed form) by at least lambda alpha_k ||z_k||^2, whenever the lower
    solves met their tolerance (so ||x~ - x^|| <= ||grad_x h|| / mu <= eps).
    One trial per (eps, alpha_0) pair, from loose accuracies (1e-2) down to
    tight ones; the sweep must contain steps that violate the decrease (which
    psi has to reject) and steps that psi accepts."""
    a, y = strongly_convex_instance(seed)
    alpha, beta = 0.05, 0.05
    P = orc.Problem(1, 12, 12, 3, alpha=alpha, reg=orc.REG_QUAD, beta=beta)

    def ell_exact(bb):
        xh = quad_lower_closed(bb, y, alpha)
        return float(np.sum((fft_conv(a, xh) - y) ** 2)) + sobolev_closed(bb, a, beta, 1.0)

    assert quad_mu(a, alpha, 12, 12) >= 1.0
    l0 = ell_exact(a)
    accepted, violating, skipped = 0, 0, 0
    for eps in (1e-2, 3e-3, 1e-3, 1e-4, 1e-5, 1e-6):
        xk, _, _ = P.fista(a, y, y, eps=eps, max_iters=100000)
        z = P.hypergrad(a, a, xk, y, eps, cg_max=20000)[0]
        zz = float(np.sum(z ** 2))
        for step in (3.0, 1.0, 0.3, 0.1, 0.03, 0.01, 0.003):
            if quad_mu(a - step * z, alpha, 12, 12) < 1.0:   # the bound on ||x~' - x^'|| needs mu >= 1
                skipped += 1
                continue
            bad = ell_exact(a - step * z) - l0 > -1e-4 * step * zz
            violating += bad
            s = P.maid_init(a, eps=eps, delta=eps, step=step, max_rounds=1, max_bt=1,
                            ll_max_iters=100000, cg_max_iters=20000)
            b, x = a.copy(), y.copy()
            acc, _ = P.maid_step(s, a, y, b, x)
            assert not s.ll_capped and s.lam == 1e-4
            assert s.znorm == pytest.approx(np.sqrt(zz), rel=1e-9)
            if acc:
                accepted += 1
                assert not bad
                assert ell_exact(b) - l0 <= -s.lam * step * s.znorm ** 2
    assert accepted >= 2 and violating >= 6 and skipped <= 15
