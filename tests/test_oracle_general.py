"""Pins of the generalised inequality (Sec. III-C, Eq. LMI_general with one
term, A~ = A(alpha)^T, B~ = I): A(alpha)^T P(alpha) + P(alpha) A(alpha) + R(alpha)
< 0, with the dual objective a chosen by the caller.

With R = C^T C and a = the svec weights of W = B B^T the SDP is the H2
analysis problem: the smallest tr(W P) over P > 0 with A^T P + P A + C^T C <= 0
is tr(B^T W_o B), W_o the observability Gramian (A^T W_o + W_o A + C^T C = 0),
i.e. the squared H2 norm of (A, B, C): a closed form from scipy's Lyapunov
solver, independent of the oracle.
"""

import numpy as np
import pytest
import scipy.linalg

from oracle import certify, ipm, polya, sdp
from paper_1411_3769_gb300 import synth


def svec_weights(W: np.ndarray) -> np.ndarray:
    """a with a^T svec(P) = tr(W P) in the basis order (unit off-diagonal entries)."""
    n = W.shape[0]
    return np.array([W[r, s] if r == s else 2.0 * W[r, s] for r, s in sdp.svec_pairs(n)])


def h2_squared(A, B, Cz):
    Wo = scipy.linalg.solve_continuous_lyapunov(A.T, -Cz.T @ Cz)
    return float(np.trace(B.T @ Wo @ B)), Wo


def _system(seed, n=4, m=2, p=2):
    rng = np.random.default_rng(seed)
    A = synth.system(n, 1, 0.0, seed)[0]
    return A, rng.normal(size=(n, m)), rng.normal(size=(p, n))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_h2_norm_is_the_sdp_optimum(seed):
    A, B, Cz = _system(seed)
    n = A.shape[0]
    h2, Wo = h2_squared(A, B, Cz)
    assert np.linalg.eigvalsh(Wo).min() > 1e-6
    a = svec_weights(B @ B.T)
    prob = sdp.Problem(A[None], 1, 0, delta=1e-9, R=(Cz.T @ Cz)[None], d_r=0, a=a)
    status, st = ipm.solve(prob, ipm.Options(eps=1e-9))
    assert status == ipm.OK
    psi = float(prob.a @ st.y)
    assert abs(psi - h2) <= 1e-6 * h2
    # the certificate of the generalised inequality holds on the final iterate
    assert certify.certify(prob, st.y)["verdict"] == 1
    assert certify.grid_check(prob, st.y, 4)["ok"]


def test_constant_term_coefficients_by_brute_force():
    """C's Lyapunov blocks are the coefficients of R(alpha) (sum alpha)^e:
    expand the product symbolically for l = 3, d_r = 1, e = 2."""
    n, l = 2, 3
    rng = np.random.default_rng(4)
    A = rng.normal(size=(l, n, n))
    R = rng.normal(size=(l, n, n))
    R = R + np.swapaxes(R, 1, 2)
    prob = sdp.Problem(A, 1, 1, R=R, d_r=1)      # degree d_p + d_a + d2 = 3, e = 2
    terms = {}
    for k, rho in enumerate(polya.monomials(l, 1)):
        for e1 in range(l):
            for e2 in range(l):
                g = list(rho)
                g[e1] += 1
                g[e2] += 1
                terms[tuple(g)] = terms.get(tuple(g), 0) + R[k]
    for j, g in enumerate(polya.monomials(l, 3)):
        ref = terms.get(tuple(g), np.zeros((n, n)))
        assert np.allclose(prob.CR[j], ref, rtol=1e-14, atol=1e-14)
        assert np.array_equal(prob.C[prob.L + j], prob.CR[j])


def test_two_vertex_bound_and_the_equal_vertex_case():
    """l = 2, d_p = 1: the optimum is at least the sum of the vertices' H2
    norms squared (P(e_i) = P_i satisfies vertex i's Lyapunov inequality), with
    equality when both vertices are the same system."""
    n = 4
    rng = np.random.default_rng(8)
    Bm = rng.normal(size=(n, 2))
    Cz = rng.normal(size=(1, n))
    a = np.concatenate([svec_weights(Bm @ Bm.T)] * 2)
    for s, equal in ((0.0, True), (0.3, False)):
        A = synth.system(n, 2, s, 5)
        prob = sdp.Problem(A, 1, 0, delta=1e-9, R=(Cz.T @ Cz)[None], d_r=0, a=a)
        status, st = ipm.solve(prob, ipm.Options(eps=1e-9))
        assert status == ipm.OK
        psi = float(prob.a @ st.y)
        vertex = sum(h2_squared(A[i], Bm, Cz)[0] for i in range(2))
        assert psi >= vertex * (1 - 1e-6)
        if equal:
            assert abs(psi - vertex) <= 1e-6 * vertex
        assert certify.certify(prob, st.y)["verdict"] == 1
        assert certify.grid_check(prob, st.y, 10)["ok"]


def test_constant_term_enters_the_certificate():
    """A P that certifies A^T P + P A < 0 fails once R exceeds its margin."""
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    status, st = ipm.solve(prob)
    cert = certify.certify(prob, st.y)
    assert cert["verdict"] == 1
    big = 2.0 * abs(cert["maxLyap_margin"]) * np.eye(w["n"])[None] * (1 + 1e-9)
    prob_r = sdp.Problem(A, w["d_p"], w["d1"], R=big * 4.0, d_r=0)
    assert certify.certify(prob_r, st.y)["verdict"] == 0
    assert not certify.grid_check(prob_r, st.y, 10)["ok"]
