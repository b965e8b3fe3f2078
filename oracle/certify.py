"""Stability certificate (oracle; test-only).

Theorem 1: x' = A(alpha) x is stable on the simplex if some P(alpha) has
P(alpha) > 0 and A^T(alpha) P(alpha) + P(alpha) A(alpha) < 0 there.
Theorem 2 (Polya), sufficient direction: a homogeneous matrix polynomial whose
coefficients are all positive definite is positive definite on the simplex.
So, with P_h recovered from y (Root step 4 of Algorithm 2), the system is
certified robustly stable when every coefficient of Eq. (LMI_3),
sum_h beta_{h,gamma} P_h, and every coefficient of Eq. (LMI_4) negated,
-sum_h (H_{h,gamma}^T P_h + P_h H_{h,gamma}), is positive definite.

Reading R-A5: a coefficient matrix M counts as positive definite when its
smallest FP64 eigenvalue exceeds tau_c(M) = 64 n u ||M||_F (u = 2^-53), a
bound on the rounding error of the symmetric eigenvalue computation.  The
verdict depends only on y, not on how the IPM stopped.

``grid_check`` evaluates the two inequalities of Theorem 1 on the simplex
lattice {gamma / N : gamma in W_N} (a necessary condition for a valid
certificate), and ``grid_max_real_eig`` is the falsifier: a lattice point with
max Re lambda(A(alpha)) >= 0 proves the system is not robustly stable.
"""

from __future__ import annotations

import numpy as np

from . import polya
from .sdp import Problem

U64 = 2.0 ** -53


def tau_c(M: np.ndarray) -> float:
    n = M.shape[0]
    return 64.0 * n * U64 * float(np.linalg.norm(M))


def coefficient_matrices(prob: Problem, y: np.ndarray):
    """The L P-side and M Lyapunov coefficient matrices built from y (with the
    generalised form's R(alpha), the Lyapunov ones are -(A^T P + P A + R))."""
    P = prob.P_from_y(y)
    coefP = np.einsum("hg,hij->gij", prob.beta.astype(np.float64), P)
    coefL = np.zeros((prob.M, prob.n, prob.n))
    for j in range(prob.M):
        acc = np.zeros((prob.n, prob.n))
        for h in range(prob.L0):
            acc += prob.H[h, j].T @ P[h] + P[h] @ prob.H[h, j]
        coefL[j] = -acc - prob.CR[j]
    return coefP, coefL


def certify(prob: Problem, y: np.ndarray) -> dict:
    coefP, coefL = coefficient_matrices(prob, y)
    lamP = np.array([np.linalg.eigvalsh(M).min() for M in coefP])
    lamL = np.array([np.linalg.eigvalsh(M).min() for M in coefL])
    okP = all(lam > tau_c(M) for lam, M in zip(lamP, coefP))
    okL = all(lam > tau_c(M) for lam, M in zip(lamL, coefL))
    return dict(verdict=int(okP and okL), minP_margin=float(lamP.min()),
                maxLyap_margin=float(-lamL.min()), lamP=lamP, lamL=lamL)


def simplex_grid(l: int, N: int) -> np.ndarray:
    return np.array(polya.monomials(l, N), dtype=np.float64) / N


def eval_poly(coefs: np.ndarray, expos, alpha: np.ndarray) -> np.ndarray:
    """sum_k coefs[k] * alpha^{expos[k]}."""
    w = np.array([np.prod(alpha ** np.array(e)) for e in expos])
    return np.einsum("k,kij->ij", w, coefs)


def grid_check(prob: Problem, y: np.ndarray, N: int) -> dict:
    P = prob.P_from_y(y)
    W0 = polya.monomials(prob.l, prob.d_p)
    Wa = polya.monomials(prob.l, prob.d_a)
    Wr = polya.monomials(prob.l, prob.d_r) if prob.R is not None else None
    minP, maxQ = np.inf, -np.inf
    for alpha in simplex_grid(prob.l, N):
        Pa = eval_poly(P, W0, alpha)
        Aa = eval_poly(prob.A, Wa, alpha)
        Q = Aa.T @ Pa + Pa @ Aa
        if Wr is not None:
            Q = Q + eval_poly(prob.R, Wr, alpha)
        minP = min(minP, np.linalg.eigvalsh(Pa).min())
        maxQ = max(maxQ, np.linalg.eigvalsh(Q).max())
    return dict(minP=float(minP), maxQ=float(maxQ), ok=bool(minP > 0 and maxQ < 0))


def grid_max_real_eig(A: np.ndarray, d_a: int, l: int, N: int) -> float:
    Wa = polya.monomials(l, d_a)
    return float(max(np.linalg.eigvals(eval_poly(A, Wa, al)).real.max()
                     for al in simplex_grid(l, N)))
