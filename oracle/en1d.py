"""FP64 oracle of the 1D elastic-net variant of ADP-beta (Sec. 4.1).

TEST INFRASTRUCTURE ONLY: the same rule as the rest of ``oracle/`` holds (only
``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` use it;
the product library shares no code with it).  Plain NumPy in float64, written
from the paper's definitions in its order:

* the operator is a full n x n matrix B (the kernel b(t, tau) of Eq. 2.4 on a
  grid), learned with beta = 0, so the upper level is l(B) = ||A x(B) - y||^2
  (Eq. 2.5a with r = 0);
* the lower level is h(x; B) = 1/2 ||B x - y||^2 + a1 ||x||_1 + a2 ||x||_2^2,
  the elastic net of Sec. 4.1, solved by proximal gradient with step lam
  (Sec. 4.1: "proximal-gradient descent method with step size lambda_x");
* Algorithm 1 (InexactGradient) and Algorithm 2 (MAID) as for the 2D problem.

Readings where the paper is silent:
* the 1/2 on the data term of h, as in the 2D readings;
* the accuracy of a lower-level iterate is the norm of the proximal-gradient
  mapping G(x) = (x - prox(x - lam grad f(x))) / lam, which equals grad h
  where h is smooth; the solve returns the first iterate whose ||G|| <= eps;
* the hypergradient differentiates the solution on its support
  S = {i : x_i != 0}: (B^T B + 2 a2 I)_SS q_S = grad g(x)_S by CG, q = 0 off
  S, and z = -((B x - y) q^T + (B q) x^T) (the mixed second derivative of h);
* L of grad g in Eq. 3.4 is bounded by 2 ||A||_1 ||A||_inf.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def prox(v, lam, a1, a2):
    """prox of lam (a1 |.| + a2 (.)^2): soft threshold at lam a1, then scale by
    1 / (1 + 2 lam a2) (the two terms act on each coordinate separately)."""
    return np.sign(v) * np.maximum(np.abs(v) - lam * a1, 0.0) / (1.0 + 2.0 * lam * a2)


def grad_map(B, y, x, lam, a1, a2):
    """Proximal-gradient mapping G(x) and the next iterate x+."""
    g = B.T @ (B @ x - y)
    xp = prox(x - lam * g, lam, a1, a2)
    return (x - xp) / lam, xp


def lower_solve(B, y, x0, eps, max_iters, lam, a1, a2):
    """Proximal gradient from x0 (Algorithm 1, step 1, with the elastic net):
    returns (x, updates made, ||G(x)||).  The first iterate whose ||G|| <= eps
    is returned; at the cap the last iterate is returned with its ||G||."""
    x = np.array(x0, dtype=np.float64, copy=True)
    k = 0
    while True:
        G, xp = grad_map(B, y, x, lam, a1, a2)
        gn = float(np.linalg.norm(G))
        if gn <= eps or k >= max_iters:
            return x, k, gn
        x = xp
        k += 1


def upper(A, x, y):
    """g(x) = ||A x - y||^2 and ||grad g(x)|| = ||2 A^T (A x - y)|| (beta = 0)."""
    e = A @ x - y
    return float(e @ e), float(np.linalg.norm(2.0 * A.T @ e))


def hypergrad(A, B, x, y, a2, delta, cg_max, rhs=None):
    """Algorithm 1, steps 2-3, on the support S of x: CG from q = 0 on
    (B^T B + 2 a2 I)_SS q_S = rhs_S (rhs = grad g(x) by default) until
    ||r|| <= delta; then z = -((B x - y) q^T + (B q) x^T).  Returns
    (z, q, iterations, ||r||, capped)."""
    S = x != 0.0
    b = 2.0 * A.T @ (A @ x - y) if rhs is None else np.asarray(rhs, dtype=np.float64)
    b = np.where(S, b, 0.0)

    def H(v):
        return np.where(S, B.T @ (B @ v) + 2.0 * a2 * v, 0.0)

    q = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    it = 0
    while np.sqrt(rr) > delta and it < cg_max:
        Hp = H(p)
        php = float(p @ Hp)
        if php <= 0.0:
            break
        a = rr / php
        q = q + a * p
        r = r - a * Hp
        rn = float(r @ r)
        p = r + (rn / rr) * p
        rr = rn
        it += 1
    res = float(np.sqrt(rr))
    z = -(np.outer(B @ x - y, q) + np.outer(B @ q, x))
    return z, q, it, res, res > delta


def L_gx(A) -> float:
    """Bound on the Lipschitz constant of grad g: 2 ||A||_2^2 <= 2 ||A||_1 ||A||_inf."""
    return 2.0 * float(np.abs(A).sum(axis=0).max()) * float(np.abs(A).sum(axis=1).max())


@dataclass
class MaidState:
    """Algorithm 2 state (Sec. 4.1's constants by default) and the last step's report."""
    eps: float = 1e-2
    delta: float = 1e-2
    step: float = 0.1
    lam_ls: float = 1e-4
    rho_up: float = 1.1
    rho_down: float = 0.5
    nu_up: float = 1.25
    nu_down: float = 0.5
    L_gx: float = 2.0
    eps_stop: float = 0.0
    max_bt: int = 5
    max_rounds: int = 20
    ll_max_iters: int = 300
    cg_max_iters: int = 1000
    k: int = 0
    accepted: int = 0
    rounds: int = 0
    trials: int = 0
    ll_iters: int = 0
    cg_iters: int = 0
    ll_capped: int = 0
    cg_capped: int = 0
    stopped: int = 0
    loss: float = 0.0
    gradx_norm: float = 0.0
    znorm: float = 0.0
    psi: float = 0.0


class Problem:
    """The 1D elastic-net ADP-beta problem (beta = 0) for a fixed A and y."""

    def __init__(self, A, y, a1=1.2e-3, a2=4e-3, lam=0.1):
        self.A = np.asarray(A, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.a1, self.a2, self.lam = a1, a2, lam

    def lower_solve(self, B, x0, eps, max_iters):
        return lower_solve(B, self.y, x0, eps, max_iters, self.lam, self.a1, self.a2)

    def upper(self, x):
        return upper(self.A, x, self.y)

    def hypergrad(self, B, x, delta, cg_max, rhs=None):
        return hypergrad(self.A, B, x, self.y, self.a2, delta, cg_max, rhs)

    def maid_init(self, **kw) -> MaidState:
        s = MaidState(L_gx=L_gx(self.A))
        for k, v in kw.items():
            setattr(s, k, v)
        return s

    def maid_step(self, s: MaidState, B, x):
        """One upper iteration of Algorithm 2 (the same control as the 2D
        oracle): B and x are updated in place on acceptance; returns accepted."""
        s.accepted = s.rounds = s.trials = s.ll_iters = s.cg_iters = 0
        s.ll_capped = s.cg_capped = s.stopped = 0
        if s.eps_stop > 0.0 and s.eps <= s.eps_stop:
            s.stopped = 1
            return False
        j = s.max_bt
        for rnd in range(s.max_rounds):
            s.rounds = rnd + 1
            xs, it, gn = self.lower_solve(B, x, s.eps, s.ll_max_iters)
            x[...] = xs
            s.ll_iters += it
            if gn > s.eps:
                s.ll_capped = 1
            l0, gx0 = self.upper(x)
            z, q, cit, res, capped = self.hypergrad(B, x, s.delta, s.cg_max_iters)
            s.cg_iters += cit
            if capped:
                s.cg_capped = 1
            zz = float((z * z).sum())
            s.znorm = float(np.sqrt(zz))
            for _ in range(j):
                s.trials += 1
                Bt = B - s.step * z
                xt, it, gn = self.lower_solve(Bt, x, s.eps, s.ll_max_iters)
                s.ll_iters += it
                if gn > s.eps:
                    s.ll_capped = 1
                l1, gx1 = self.upper(xt)
                eb = s.eps         # eps_bar_{k+1} = eps_k, as in the 2D reading
                psi = l1 + gx1 * eb + 0.5 * s.L_gx * eb * eb - l0 + gx0 * eb + s.lam_ls * s.step * zz
                s.psi = psi
                if psi <= 0.0:
                    B[...] = Bt
                    x[...] = xt
                    s.loss, s.gradx_norm = l1, gx1
                    s.eps *= s.nu_up
                    s.delta *= s.nu_up
                    s.step *= s.rho_up
                    s.k += 1
                    s.accepted = 1
                    return True
                s.step *= s.rho_down
            j += 1
            s.loss, s.gradx_norm = l0, gx0
            s.eps *= s.nu_down
            s.delta *= s.nu_down
            if s.eps_stop > 0.0 and s.eps <= s.eps_stop:
                s.stopped = 1
                break
        return False
