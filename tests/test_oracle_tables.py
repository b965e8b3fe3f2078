"""Pins of the oracle's Polya tables (Sec. I notation, Sec. II, Sec. III-A)."""

import itertools
from math import comb, factorial

import numpy as np
import pytest

from oracle import polya
from tests.conftest import golden


def test_monomial_order_matches_homogenisation_example():
    # Sec. II example lists B_1..B_6 for a1^2, a1a2, a1a3, a2^2, a2a3, a3^2
    rows = golden("homogenization_example.txt")
    W2 = polya.monomials(3, 2)
    for r in rows:
        idx, g = int(r[0]), tuple(int(x) for x in r[1:4])
        assert W2[idx - 1] == g
        assert polya.lex_index(g) == idx


@pytest.mark.parametrize("l,d", [(1, 3), (2, 2), (3, 2), (3, 4), (4, 3), (5, 2)])
def test_lex_index_is_rank_and_printed_formula_is_reversed(l, d):
    W = polya.monomials(l, d)
    assert len(W) == polya.f_card(l, d) == len(set(W))
    # strictly decreasing lexicographically: leftmost non-zero of g - h positive
    for g, h in zip(W, W[1:]):
        diff = [a - b for a, b in zip(g, h)]
        assert next(x for x in diff if x != 0) > 0
    for k, g in enumerate(W):
        assert polya.lex_index(g) == k + 1
        # Eq. (1) as printed ranks in the opposite order (reading R-A1)
        assert polya.printed_lex_index(g) == len(W) - k


def test_beta_worked_example():
    for l, d_p, d1, h, g, val in golden("beta_example.txt"):
        beta = polya.beta_table(int(l), int(d_p), int(d1))
        assert beta[int(h) - 1, int(g) - 1] == int(val)


def test_H_worked_example():
    for l, d_p, d_a, d2, h, g, c1, c2 in golden("H_example.txt"):
        c = polya.h_coeff_table(int(l), int(d_p), int(d_a), int(d2))
        assert list(c[int(h) - 1, int(g) - 1]) == [int(c1), int(c2)]


def test_homogenisation_worked_example():
    # tags: C, D, E, F as unit vectors of R^4
    C, D, E, F = np.eye(4)
    terms = {(2, 0, 0): C, (0, 1, 0): D, (0, 0, 1): E, (0, 0, 0): F}
    out = polya.homogenize(terms, 3)
    W2 = polya.monomials(3, 2)
    for r in golden("homogenization_example.txt"):
        g = W2[int(r[0]) - 1]
        assert np.array_equal(out[g], np.array(r[4:8]))


CASES = [(l, dp, d1) for l in (1, 2, 3, 4) for dp in (0, 1, 2, 3) for d1 in (0, 1, 2, 4)]


@pytest.mark.parametrize("l,d_p,d1", CASES)
def test_beta_closed_form_and_identities(l, d_p, d1):
    beta = polya.beta_table(l, d_p, d1)
    W0, W = polya.monomials(l, d_p), polya.monomials(l, d_p + d1)
    for hi, h in enumerate(W0):
        for gi, g in enumerate(W):
            assert beta[hi, gi] == polya.multinomial(d1, [a - b for a, b in zip(g, h)])
    # each P_h is spread over (sum alpha)^{d1}: its coefficients sum to l^{d1}
    assert np.all(beta.sum(axis=1) == l ** d1)
    # sum_h beta_{h,gamma} d_p!/h! = (d_p+d1)!/gamma!  (so C_gamma = delta*multinomial*I)
    w = np.array([polya.multinomial(d_p, h) for h in W0])
    for gi, g in enumerate(W):
        assert int(w @ beta[:, gi]) == polya.multinomial(d_p + d1, g)


@pytest.mark.parametrize("l,d_p,d_a,d2", [(2, 1, 1, 1), (3, 2, 1, 3), (3, 1, 2, 2), (4, 2, 1, 2), (2, 0, 3, 2)])
def test_H_closed_form(l, d_p, d_a, d2):
    c = polya.h_coeff_table(l, d_p, d_a, d2)
    W0, Wa, W = polya.monomials(l, d_p), polya.monomials(l, d_a), polya.monomials(l, d_p + d_a + d2)
    for hi, h in enumerate(W0):
        for gi, g in enumerate(W):
            for li, lam in enumerate(Wa):
                mu = [g[m] - h[m] - lam[m] for m in range(l)]
                assert c[hi, gi, li] == polya.multinomial(d2, mu)


def _poly_mul(p, q):
    out = {}
    for e1, c1 in p.items():
        for e2, c2 in q.items():
            e = tuple(a + b for a, b in zip(e1, e2))
            out[e] = out.get(e, 0) + c1 * c2
    return out


@pytest.mark.parametrize("l,d_p,d1", [(2, 1, 1), (2, 2, 3), (3, 1, 2), (3, 2, 2), (4, 1, 1)])
def test_beta_brute_force_expansion(l, d_p, d1):
    # expand (sum alpha)^{d1} * P(alpha) with P_h as symbolic unit tags
    W0 = polya.monomials(l, d_p)
    P = {h: np.eye(len(W0), dtype=np.int64)[k] for k, h in enumerate(W0)}
    s = {tuple(1 if m == k else 0 for m in range(l)): 1 for k in range(l)}
    poly = P
    for _ in range(d1):
        poly = _poly_mul(s, poly)
    beta = polya.beta_table(l, d_p, d1)
    for gi, g in enumerate(polya.monomials(l, d_p + d1)):
        assert np.array_equal(poly.get(g, 0) * np.ones(len(W0), dtype=np.int64), beta[:, gi])


@pytest.mark.parametrize("l,d_p,d2", [(2, 1, 1), (3, 1, 2), (3, 2, 1), (2, 2, 3)])
def test_H_brute_force_expansion(l, d_p, d2):
    # expand (sum alpha)^{d2} * (A(alpha)^T P(alpha) + P(alpha) A(alpha)) keeping the
    # products A_lambda-with-P_h as integer tags (h, lambda); the coefficient of the tag
    # in monomial gamma is the number of times H_{h,gamma} contains A_lambda.
    W0, Wa = polya.monomials(l, d_p), polya.monomials(l, 1)
    L0, Na = len(W0), len(Wa)
    PA = {}
    for hi, h in enumerate(W0):
        for li, lam in enumerate(Wa):
            e = tuple(a + b for a, b in zip(h, lam))
            tag = np.zeros((L0, Na), dtype=np.int64)
            tag[hi, li] = 1
            PA[e] = PA.get(e, 0) + tag
    s = {tuple(1 if m == k else 0 for m in range(l)): 1 for k in range(l)}
    poly = PA
    for _ in range(d2):
        poly = _poly_mul(s, poly)
    c = polya.h_coeff_table(l, d_p, 1, d2)
    for gi, g in enumerate(polya.monomials(l, d_p + 1 + d2)):
        assert np.array_equal(poly.get(g, np.zeros((L0, Na), dtype=np.int64)), c[:, gi, :])


@pytest.mark.parametrize("name,n,l,d_p,d1,expect", [
    ("tiny", 5, 2, 1, 1, dict(L0=2, L=3, M=4, K=30, nblk=7)),
    ("mid", 20, 4, 2, 3, dict(L0=10, L=56, M=84, K=2100, nblk=140)),
    ("large", 100, 3, 2, 4, dict(L0=6, L=28, M=36, K=30300, nblk=64)),
    ("warm", 32, 3, 2, 3, dict(L0=6, L=21, M=28, K=3168, nblk=49)),
    # Example 1 of Sec. V: 224 constraints, X of order 1092 (n=7, l=8, d_p=1, d1=d2=1)
    ("tokamak", 7, 8, 1, 1, dict(L0=8, K=224, nblk=156)),
])
def test_counts(name, n, l, d_p, d1, expect):
    sz = polya.sizes(n, l, d_p, d1)
    for k, v in expect.items():
        assert sz[k] == v, (name, k)
    if name == "tokamak":
        assert sz["nblk"] * n == 1092


def test_f_card_formula():
    for l in range(1, 7):
        for d in range(0, 7):
            assert polya.f_card(l, d) == comb(l + d - 1, l - 1)
            assert polya.f_card(l, d) == sum(1 for g in itertools.product(range(d + 1), repeat=l) if sum(g) == d)
    assert polya.f_card(0, 3) == 0


def test_multinomial():
    assert polya.multinomial(4, (2, 1, 1)) == factorial(4) // 2
    assert polya.multinomial(3, (2, 2)) == 0
    assert polya.multinomial(3, (4, -1)) == 0
