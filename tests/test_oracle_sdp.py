"""Pins of the oracle's SDP elements and Schur complement (Sec. III-B, Sec. IV)."""

import numpy as np
import pytest

from oracle import polya, sdp
from paper_1411_3769_gb300 import synth


def _prob(n=4, l=3, d_p=1, d1=2, s=0.5, seed=0, d2=None, d_a=1):
    if d_a == 1:
        A = synth.system(n, l, s, seed)
    else:
        rng = np.random.default_rng(seed)
        A = rng.normal(size=(polya.f_card(l, d_a), n, n))
    return sdp.Problem(A, d_p, d1, d2=d2, d_a=d_a)


def _spd_blocks(rng, nblk, n):
    G = rng.normal(size=(nblk, n, n))
    return np.einsum("gij,gkj->gik", G, G) + n * np.eye(n)


def test_basis_spans_symmetric_matrices():
    for n in (1, 2, 5, 7):
        Nt = n * (n + 1) // 2
        E = np.stack([sdp.basis_matrix(n, k) for k in range(Nt)])
        assert np.allclose(E, np.swapaxes(E, 1, 2))
        G = np.einsum("aij,bij->ab", E, E)
        assert np.linalg.matrix_rank(G) == Nt
        # first n are the diagonal units, the next n-1 the first superdiagonal (Sec. I)
        for k in range(n):
            assert E[k][k, k] == 1 and E[k].sum() == 1
        for k in range(n - 1):
            assert E[n + k][k, k + 1] == 1 and E[n + k].sum() == 2


def test_smat_svec_adjoint():
    rng = np.random.default_rng(1)
    n = 5
    v = rng.normal(size=15)
    W = rng.normal(size=(n, n))
    assert np.isclose(np.trace(sdp.smat(v, n) @ W), v @ sdp.svec_adjoint(W))


@pytest.mark.parametrize("kw", [dict(), dict(d_p=2, d1=1), dict(l=2, d_p=0, d1=3), dict(d_a=2, l=2, d1=1, d_p=1),
                                dict(d2=3, d1=1)])
def test_BT_and_B_match_literal_elements(kw):
    prob = _prob(**kw)
    B = prob.literal_B()
    rng = np.random.default_rng(2)
    v = rng.normal(size=prob.K)
    assert np.allclose(prob.BT(v), np.einsum("i,igab->gab", v, B), atol=1e-12)
    W = rng.normal(size=(prob.nblk, prob.n, prob.n))
    assert np.allclose(prob.Bop(W), np.einsum("igab,gba->i", B, W), atol=1e-12)
    # adjoint pair: <B^T(v), W> = <v, B(W)>
    assert np.isclose(np.sum(prob.BT(v) * W), v @ prob.Bop(W))
    # every B_i is symmetric and block diagonal by construction (Eq. Ai)
    assert np.allclose(B, np.swapaxes(B, -1, -2))


@pytest.mark.parametrize("kw", [dict(n=3, l=2, d_p=1, d1=1), dict(n=3, l=3, d_p=2, d1=1), dict(n=2, l=2, d_p=2, d1=2, d_a=2)])
def test_BT_is_polya_expansion(kw):
    """B^T(y) P-side blocks are the coefficients of (sum a)^{d1} P(a) (Eq. LMI_3);
    Lyapunov blocks are the coefficients of -(sum a)^{d2}(A^T P + P A) (Eq. LMI_4).
    Checked by evaluating both polynomials at random simplex points."""
    prob = _prob(**kw)
    rng = np.random.default_rng(3)
    y = rng.normal(size=prob.K)
    S = prob.BT(y)
    P = prob.P_from_y(y)
    W0 = polya.monomials(prob.l, prob.d_p)
    Wa = polya.monomials(prob.l, prob.d_a)
    WL = polya.monomials(prob.l, prob.d_p + prob.d1)
    WM = polya.monomials(prob.l, prob.d_p + prob.d_a + prob.d2)

    def ev(coefs, expos, al):
        return sum(c * np.prod(al ** np.array(e)) for c, e in zip(coefs, expos))
    for _ in range(5):
        al = rng.random(prob.l)
        Pa, Aa = ev(P, W0, al), ev(prob.A, Wa, al)
        lhs1 = al.sum() ** prob.d1 * Pa
        assert np.allclose(lhs1, ev(S[:prob.L], WL, al), atol=1e-10)
        lhs2 = -(al.sum() ** prob.d2) * (Aa.T @ Pa + Pa @ Aa)
        assert np.allclose(lhs2, ev(S[prob.L:], WM, al), atol=1e-10)


def test_C_blocks():
    prob = _prob(n=3, l=3, d_p=2, d1=2)
    WL = polya.monomials(3, 4)
    for j, g in enumerate(WL):
        assert np.allclose(prob.C[j], polya.multinomial(4, g) * np.eye(3))
    assert np.all(prob.C[prob.L:] == 0)


@pytest.mark.parametrize("kw", [dict(n=3, l=2, d_p=1, d1=1), dict(n=3, l=3, d_p=2, d1=1),
                                dict(n=4, l=2, d_p=1, d1=2), dict(n=2, l=2, d_p=1, d1=1, d_a=2),
                                dict(n=3, l=2, d_p=0, d1=2)])
def test_schur_structured_matches_definition(kw):
    prob = _prob(**kw)
    rng = np.random.default_rng(4)
    X = _spd_blocks(rng, prob.nblk, prob.n)
    Z = _spd_blocks(rng, prob.nblk, prob.n)
    Y = np.linalg.inv(Z)
    Ol = prob.schur_literal(Y, X)
    Os = prob.schur_structured(Y, X)
    assert np.abs(Ol - Os).max() <= 1e-13 * np.abs(Ol).max()
    # symmetric positive definite (B_i linearly independent)
    assert np.allclose(Os, Os.T, rtol=0, atol=1e-12 * np.abs(Os).max())
    assert np.linalg.eigvalsh(0.5 * (Os + Os.T)).min() > 0
    # matrix-free identity Omega v = B(Z^{-1} B^T(v) X)
    v = rng.normal(size=prob.K)
    assert np.allclose(Os @ v, prob.schur_matvec(Y, X, v), rtol=1e-12, atol=1e-12 * np.abs(Os).max())


def test_schur_terms_catch_transposition():
    """A plausible slip (a transposed H in one of the four Lyapunov terms) is
    visible: the structured formula then disagrees with the definition."""
    prob = _prob(n=3, l=2, d_p=1, d1=1, s=0.7)
    rng = np.random.default_rng(5)
    X = _spd_blocks(rng, prob.nblk, prob.n)
    Y = np.linalg.inv(_spd_blocks(rng, prob.nblk, prob.n))
    good = prob.schur_structured(Y, X)
    orig = prob.schur_terms

    def bad_terms(a, b, Y_, X_):
        t = orig(a, b, Y_, X_)
        Ps, Ph = t[-1]
        t[-1] = (Ps.T, Ph)
        return t
    prob.schur_terms = bad_terms
    try:
        bad = prob.schur_structured(Y, X)
    finally:
        prob.schur_terms = orig
    assert np.abs(bad - good).max() > 1e-6 * np.abs(good).max()
