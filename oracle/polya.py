"""Monomials, index map and the Polya coefficient tables (oracle; test-only).

Follows Sec. I "Notation" and Sec. III-A of the paper.

* W_d is the set of exponents gamma in N^l with |gamma| = d, totally ordered
  lexicographically: gamma precedes eta when the leftmost non-zero entry of
  gamma - eta is positive.  So (d,0,...,0) comes first.  The closed-form rank
  printed as Eq. (1) counts the other way round (it places (0,...,0,d) first);
  ``printed_lex_index`` restates it so a test can show the reversal, and the
  oracle uses the order of the text and of both worked examples.
* beta_{h,gamma} (Eqs. beta_init, beta) is the scalar multiplying P_h in the
  alpha^gamma coefficient of (sum_i alpha_i)^{d_1} P(alpha).
* H_{h,gamma} (Eqs. H_init, H) is the matrix multiplying P_h (left-transposed
  and right) in the alpha^gamma coefficient of
  (sum_i alpha_i)^{d_2} (A^T P + P A).  Because every step of its recursion is
  a sum of the A_lambda, H_{h,gamma} = sum_lambda c[h,gamma,lambda] A_lambda
  with integer c; the oracle carries the integer c through the recursion and
  forms the matrices from it.
"""

from __future__ import annotations

from math import comb, factorial

import numpy as np


def f_card(l: int, d: int) -> int:
    """Eq. (2): number of l-variate monomials of degree d."""
    if l == 0:
        return 0
    if d < 0:
        return 0
    return comb(l + d - 1, l - 1)


def monomials(l: int, d: int) -> list[tuple[int, ...]]:
    """W_d in the paper's lexicographic order ((d,0,...,0) first)."""
    if l <= 0 or d < 0:
        return []
    if l == 1:
        return [(d,)]
    out = []
    for g0 in range(d, -1, -1):
        for rest in monomials(l - 1, d - g0):
            out.append((g0,) + rest)
    return out


def lex_index(gamma) -> int:
    """1-based rank <gamma> of gamma within W_{|gamma|} in the text's order.

    Counts the monomials that precede gamma: for each position j, those that
    agree with gamma before j and have a larger j-th exponent.
    """
    gamma = tuple(int(g) for g in gamma)
    l = len(gamma)
    rem = sum(gamma)
    rank = 0
    for j in range(l - 1):
        for bigger in range(gamma[j] + 1, rem + 1):
            rank += f_card(l - j - 1, rem - bigger)
        rem -= gamma[j]
    return rank + 1


def printed_lex_index(gamma) -> int:
    """Eq. (1) exactly as printed (it ranks in the reverse order of the text)."""
    gamma = tuple(int(g) for g in gamma)
    l = len(gamma)
    d = sum(gamma)
    total = 0
    for j in range(1, l):
        prefix = sum(gamma[: j - 1])
        for i in range(1, gamma[j - 1] + 1):
            total += f_card(l - j, d + 1 - prefix - i)
    return total + 1


def beta_table(l: int, d_p: int, d1: int) -> np.ndarray:
    """beta[h, gamma] (0-based indices) by the recursion of Eqs. beta_init/beta.

    Shape (L0, L) with L0 = card W_{d_p}, L = card W_{d_p+d1}.
    """
    W0 = monomials(l, d_p)
    L0 = len(W0)
    # beta^(0): identity on W_{d_p}
    cur_list = W0
    cur = {g: np.array([1 if h == g else 0 for h in W0], dtype=np.int64) for g in W0}
    for i in range(1, d1 + 1):
        nxt_list = monomials(l, d_p + i)
        nxt = {}
        for g in nxt_list:
            acc = np.zeros(L0, dtype=np.int64)
            for k in range(l):  # lambda = e_k in W_1
                if g[k] == 0:
                    continue
                prev = tuple(g[m] - (1 if m == k else 0) for m in range(l))
                acc = acc + cur[prev]
            nxt[g] = acc
        cur, cur_list = nxt, nxt_list
    return np.stack([cur[g] for g in cur_list], axis=1)  # (L0, L)


def h_coeff_table(l: int, d_p: int, d_a: int, d2: int) -> np.ndarray:
    """Integer c[h, gamma, lambda] with H_{h,gamma} = sum_lambda c A_lambda.

    Recursion of Eqs. H_init/H; h in W_{d_p}, gamma in W_{d_p+d_a+d2},
    lambda in W_{d_a}.  Shape (L0, M, N_a).
    """
    W0 = monomials(l, d_p)
    Wa = monomials(l, d_a)
    L0, Na = len(W0), len(Wa)
    start = monomials(l, d_p + d_a)
    cur = {}
    for g in start:
        c0 = np.zeros((L0, Na), dtype=np.int64)
        for hi, h in enumerate(W0):
            for li, lam in enumerate(Wa):
                if all(lam[m] + h[m] == g[m] for m in range(l)):
                    c0[hi, li] += 1
        cur[g] = c0
    cur_list = start
    for i in range(1, d2 + 1):
        nxt_list = monomials(l, d_p + d_a + i)
        nxt = {}
        for g in nxt_list:
            acc = np.zeros((L0, Na), dtype=np.int64)
            for k in range(l):
                if g[k] == 0:
                    continue
                prev = tuple(g[m] - (1 if m == k else 0) for m in range(l))
                acc = acc + cur[prev]
            nxt[g] = acc
        cur, cur_list = nxt, nxt_list
    return np.stack([cur[g] for g in cur_list], axis=1)  # (L0, M, Na)


def h_matrices(c: np.ndarray, A: np.ndarray) -> np.ndarray:
    """H[h, gamma] = sum_lambda c[h,gamma,lambda] A[lambda]  -> (L0, M, n, n)."""
    return np.einsum("hgl,lij->hgij", c.astype(np.float64), A)


def multinomial(d: int, mu) -> int:
    """d! / prod(mu_i!) when mu >= 0 and |mu| = d, else 0."""
    mu = [int(m) for m in mu]
    if any(m < 0 for m in mu) or sum(mu) != d:
        return 0
    out = factorial(d)
    for m in mu:
        out //= factorial(m)
    return out


def homogenize(terms: dict, l: int) -> dict:
    """Sec. II: make A(alpha) homogeneous on the simplex.

    ``terms`` maps an exponent tuple to a coefficient (scalar or array).  Each
    monomial of degree d_i < d_a is multiplied by (sum_j alpha_j)^{d_a - d_i};
    the result maps exponents in W_{d_a} to coefficients.
    """
    d_a = max(sum(k) for k in terms)
    out: dict = {}
    for expo, coef in terms.items():
        extra = d_a - sum(expo)
        for mu in monomials(l, extra):
            w = multinomial(extra, mu)
            g = tuple(expo[m] + mu[m] for m in range(l))
            out[g] = out.get(g, 0) + w * np.asarray(coef, dtype=np.float64)
    return out


def substitute_linear(terms: dict, M) -> dict:
    """A(M alpha) for A(beta) = sum_gamma A_gamma beta^gamma (Sec. V, Examples 1
    and 2 pose the uncertainty set as the image of the simplex under a map g
    and certify A'(alpha) = A(g(alpha)) on the simplex).

    ``terms`` maps exponent tuples to coefficients; M is l x l, beta_i =
    sum_j M_ij alpha_j, so a homogeneous A of degree d stays homogeneous of
    degree d.  Each beta^gamma is expanded factor by factor (brute-force
    polynomial multiplication).
    """
    M = np.asarray(M, dtype=np.float64)
    l = M.shape[0]
    out: dict = {}
    for expo, coef in terms.items():
        poly = {tuple([0] * l): 1.0}
        for i in range(l):
            for _ in range(expo[i]):
                nxt: dict = {}
                for e, v in poly.items():
                    for j in range(l):
                        if M[i, j] == 0.0:
                            continue
                        e2 = tuple(e[k] + (1 if k == j else 0) for k in range(l))
                        nxt[e2] = nxt.get(e2, 0.0) + v * M[i, j]
                poly = nxt
        for e, v in poly.items():
            out[e] = out.get(e, 0) + v * np.asarray(coef, dtype=np.float64)
    return out


def sizes(n: int, l: int, d_p: int, d1: int, d2: int | None = None, d_a: int = 1) -> dict:
    """Eqs. (L0), (L), (M), (K): the SDP's dimensions."""
    if d2 is None:
        d2 = d1
    L0 = f_card(l, d_p)
    L = f_card(l, d_p + d1)
    M = f_card(l, d_p + d_a + d2)
    Nt = n * (n + 1) // 2
    return dict(L0=L0, L=L, M=M, Ntil=Nt, K=L0 * Nt, nblk=L + M, Na=f_card(l, d_a))
