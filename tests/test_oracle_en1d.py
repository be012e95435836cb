"""Pins of the 1D elastic-net oracle (Sec. 4.1) against what the mathematics
fixes, independently of the oracle's own formulas:

* the prox is the minimiser of its 1D objective (brute force on a fine grid);
* with B = I the lower level is separable and has a closed form;
* with a1 = 0 it is ridge regression (a library linear solve);
* at the returned solution the subdifferential optimality (KKT) conditions hold;
* the support CG equals a direct solve of the restricted system, and its n-th
  iterate minimises the energy error over the Krylov space;
* the hypergradient equals central finite differences of l(B) = ||A x(B) - y||^2
  whenever the support is stable;
* MAID's accepted steps decrease the exactly solved upper loss by lambda alpha ||z||^2
  (Lemma 1) at tight accuracies, and its psi has the Eq. 3.4 decomposition.
"""
import numpy as np
import pytest

from oracle import en1d
from paper_2502_09758_gb300 import synth

A1, A2, LAM = 1.2e-3, 4e-3, 0.1


def well_conditioned(n, seed):
    """B = (A + I) / 2 for the Gaussian A: ||B|| <= 1, smallest singular value >= ~0.5."""
    return 0.5 * (synth.gaussian_conv_matrix(n, 2.0) + np.eye(n))


@pytest.mark.parametrize("lam,a1,a2", [(0.1, 1.2e-3, 4e-3), (0.5, 0.3, 0.2), (1.0, 0.05, 0.0)])
def test_prox_is_the_minimiser(lam, a1, a2):
    rng = np.random.default_rng(1)
    v = rng.uniform(-1, 1, 40)
    p = en1d.prox(v, lam, a1, a2)
    grid = np.linspace(-1.5, 1.5, 300001)
    for vi, pi in zip(v, p):
        f = 0.5 * (grid - vi) ** 2 + lam * (a1 * np.abs(grid) + a2 * grid ** 2)
        assert abs(grid[np.argmin(f)] - pi) <= 2e-5


def test_identity_operator_closed_form():
    rng = np.random.default_rng(2)
    n = 64
    y = rng.uniform(-0.01, 0.01, n)
    x, it, gn = en1d.lower_solve(np.eye(n), y, np.zeros(n), 1e-13, 100000, LAM, A1, A2)
    exact = np.sign(y) * np.maximum(np.abs(y) - A1, 0.0) / (1.0 + 2.0 * A2)
    assert gn <= 1e-13
    assert np.max(np.abs(x - exact)) <= 1e-13
    assert (x == 0).sum() == (exact == 0).sum() > 0     # some coordinates are thresholded to zero


def test_ridge_case_is_a_linear_solve():
    rng = np.random.default_rng(3)
    n = 48
    B = well_conditioned(n, 3)
    y = rng.standard_normal(n)
    x, it, gn = en1d.lower_solve(B, y, np.zeros(n), 1e-12, 100000, LAM, 0.0, A2)
    exact = np.linalg.solve(B.T @ B + 2 * A2 * np.eye(n), B.T @ y)
    assert np.linalg.norm(x - exact) <= 1e-10 * np.linalg.norm(exact)


def test_solution_satisfies_kkt():
    rng = np.random.default_rng(4)
    n = 64
    B = well_conditioned(n, 4)
    y = 0.05 * rng.standard_normal(n)
    a1 = 0.02
    x, it, gn = en1d.lower_solve(B, y, np.zeros(n), 1e-12, 100000, LAM, a1, A2)
    g = B.T @ (B @ x - y)
    on = x != 0
    assert 0 < on.sum() < n
    assert np.max(np.abs(g[on] + a1 * np.sign(x[on]) + 2 * A2 * x[on])) <= 1e-10
    assert np.max(np.abs(g[~on])) <= a1 + 1e-10


def test_returns_first_iterate_meeting_eps_and_caps():
    rng = np.random.default_rng(5)
    n = 32
    B = well_conditioned(n, 5)
    y = 0.05 * rng.standard_normal(n)
    x, it, gn = en1d.lower_solve(B, y, np.zeros(n), 1e-3, 100000, LAM, A1, A2)
    assert gn <= 1e-3
    assert abs(np.linalg.norm(en1d.grad_map(B, y, x, LAM, A1, A2)[0]) - gn) <= 1e-15   # the norm is the point's own
    xm, itm, gnm = en1d.lower_solve(B, y, np.zeros(n), 0.0, it - 1, LAM, A1, A2)
    assert itm == it - 1 and gnm > 1e-3          # the iterate before did not meet eps
    xc, itc, gnc = en1d.lower_solve(B, y, np.zeros(n), 0.0, 7, LAM, A1, A2)
    assert itc == 7 and gnc > 0.0


def test_support_cg_matches_restricted_solve_and_krylov():
    rng = np.random.default_rng(6)
    n = 12
    A = synth.gaussian_conv_matrix(n, 1.5)
    B = well_conditioned(n, 6)
    y = rng.standard_normal(n)
    x = rng.standard_normal(n)
    x[[1, 4, 7]] = 0.0
    S = x != 0
    H = (B.T @ B + 2 * A2 * np.eye(n))[np.ix_(S, S)]
    rhs = 2 * A.T @ (A @ x - y)
    z, q, it, res, capped = en1d.hypergrad(A, B, x, y, A2, 1e-14, 1000)
    assert not capped
    assert np.allclose(q[S], np.linalg.solve(H, rhs[S]), rtol=0, atol=1e-12)
    assert np.all(q[~S] == 0.0)
    # n-th iterate: minimiser of the H-norm error over span{r0, H r0, ...}
    qs = np.linalg.solve(H, rhs[S])
    for m in (1, 2, 3):
        _, qm, itm, _, _ = en1d.hypergrad(A, B, x, y, A2, 0.0, m)
        K = np.stack([np.linalg.matrix_power(H, k) @ rhs[S] for k in range(m)], axis=1)
        Q, _ = np.linalg.qr(K)
        c = np.linalg.solve(Q.T @ H @ Q, Q.T @ rhs[S])
        assert itm == m
        assert np.linalg.norm(qm[S] - Q @ c) <= 1e-10 * np.linalg.norm(qs)


def test_hypergradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    n = 8
    A = synth.gaussian_conv_matrix(n, 1.0)
    B = well_conditioned(n, 7) + 0.05 * rng.standard_normal((n, n))
    xt = np.array([0.0, 0.8, 0.8, 0.0, 0.0, 0.5, 0.0, 0.9])
    y = A @ xt + 0.01 * rng.standard_normal(n)
    a1 = 0.01
    P = en1d.Problem(A, y, a1=a1, a2=A2, lam=0.5)

    def solve(Bm):
        x, _, gn = P.lower_solve(Bm, np.zeros(n), 1e-14, 200000)
        assert gn <= 1e-14
        return x

    x = solve(B)
    S = x != 0
    assert 0 < S.sum() < n
    z, q, it, res, capped = P.hypergrad(B, x, 1e-14, 1000)
    h = 1e-6
    for i, j in [(0, 1), (2, 5), (5, 5), (7, 3), (3, 0), (1, 7)]:
        E = np.zeros((n, n))
        E[i, j] = h
        xp, xm = solve(B + E), solve(B - E)
        assert np.array_equal(xp != 0, S) and np.array_equal(xm != 0, S)
        fd = (P.upper(xp)[0] - P.upper(xm)[0]) / (2 * h)
        assert abs(fd - z[i, j]) <= 1e-6 * max(1.0, np.abs(z).max()), (i, j, fd, z[i, j])


def tiny_instance(seed):
    s = synth.signal1d(48, seed=seed)
    return en1d.Problem(s.A, s.y, a1=A1, a2=A2, lam=LAM), s


def test_maid_lemma1_and_psi_decomposition():
    P, s = tiny_instance(8)
    B = s.A.copy()
    x = s.y.copy()
    st = P.maid_init(eps=1e-9, delta=1e-9, step=1.0, ll_max_iters=200000, cg_max_iters=10000)
    accepted = 0
    for _ in range(6):
        B0, x0 = B.copy(), x.copy()
        eps = st.eps
        acc = P.maid_step(st, B, x)
        if not acc:
            continue
        accepted += 1
        # exact upper losses at the two operators
        xe0, _, _ = P.lower_solve(B0, x0, 1e-12, 400000)
        xe1, _, _ = P.lower_solve(B, x, 1e-12, 400000)
        l0, l1 = P.upper(xe0)[0], P.upper(xe1)[0]
        step = st.step / st.rho_up
        assert l1 - l0 <= -st.lam_ls * step * st.znorm ** 2 + 1e-8
        # psi as reported = l(b') - l(b) + slack + lambda alpha ||z||^2 (Eq. 3.4),
        # l(b) and its gradient norm at the round's own solve from x0
        if st.rounds == 1:
            xr, _, _ = P.lower_solve(B0, x0, eps, st.ll_max_iters)
            lr, gr = P.upper(xr)
            slack = (st.gradx_norm + gr) * eps + 0.5 * st.L_gx * eps * eps
            assert abs(st.psi - (st.loss - lr + slack + st.lam_ls * step * st.znorm ** 2)) <= 1e-12
    assert accepted >= 2


def test_L_bounds_the_gradient_lipschitz_constant():
    A = synth.gaussian_conv_matrix(100, 5.0)
    assert en1d.L_gx(A) >= 2 * np.linalg.norm(A, 2) ** 2
