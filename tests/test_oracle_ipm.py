"""Pins of the oracle's interior-point method and certificate (Sec. IV, Thms 1-3)."""

import numpy as np
import pytest
import scipy.linalg

from oracle import certify, ipm, polya, sdp
from paper_1411_3769_gb300 import synth


def _solve(A, d_p, d1, **kw):
    prob = sdp.Problem(A, d_p, d1)
    status, st = ipm.solve(prob, ipm.Options(**kw))
    return prob, status, st


def test_newton_system_identities():
    prob = sdp.Problem(synth.system(4, 3, 0.4, 7), 1, 2)
    st = ipm.start_point(prob)
    for _ in range(3):          # a few steps in, so X, Z are not the identity
        ipm.newton_step(prob, st, ipm.Options())
    X, Z, y = st.X.copy(), st.Z.copy(), st.y.copy()
    info = ipm.newton_step(prob, st, ipm.Options())
    G = prob.C - prob.BT(y) + Z
    scale = 1 + np.abs(prob.Bop(X)).max()
    # predictor: B(X + dXh) = a  (the reading R-A7 makes this hold)
    assert np.abs(prob.Bop(X + info["dXh"]) - prob.a).max() < 1e-10 * scale
    # predictor: dZh - B^T(dyh) = -G
    assert np.abs(info["dZh"] - prob.BT(info["dyh"]) + G).max() < 1e-12 * (1 + np.abs(G).max())
    # corrector: B(dXb) = 0 and dZb = B^T(dyb)
    assert np.abs(prob.Bop(info["dXb"])).max() < 1e-10 * scale
    assert np.allclose(info["dZb"], prob.BT(info["dyb"]))
    # complementarity of the predictor: Z dXh + dZh X = -Z X, up to symmetrisation
    lhs = np.einsum("gab,gbc->gac", Z, info["dXh"]) + np.einsum("gab,gbc->gac", info["dZh"], X)
    rhs = -np.einsum("gab,gbc->gac", Z, X)
    Yi = info["Y"]
    # Y (lhs - rhs) is antisymmetric-only: its symmetric part vanishes
    D = np.einsum("gab,gbc->gac", Yi, lhs - rhs)
    assert np.abs(D + np.swapaxes(D, 1, 2)).max() < 1e-9 * (1 + np.abs(X).max())
    # the step keeps X and Z positive definite
    assert all(np.linalg.eigvalsh(b).min() > 0 for b in st.X)
    assert all(np.linalg.eigvalsh(b).min() > 0 for b in st.Z)


def test_thm3_block_structure_is_invariant():
    """Dense-mode iteration (no block structure assumed) stays block diagonal
    with the exact blocks of the block-mode iteration (Theorem 3)."""
    prob = sdp.Problem(synth.system(3, 2, 0.3, 1), 1, 1)
    n, nb = prob.n, prob.nblk
    dense = ipm.dense_solve_steps(prob, 4)
    st = ipm.start_point(prob)
    for k in range(4):
        ipm.newton_step(prob, st, ipm.Options())
        Xd, Zd, yd = dense[k]
        mask = np.kron(np.eye(nb), np.ones((n, n))) == 0
        assert np.all(Xd[mask] == 0.0) and np.all(Zd[mask] == 0.0)
        Xb = np.stack([Xd[g * n:(g + 1) * n, g * n:(g + 1) * n] for g in range(nb)])
        assert np.allclose(Xb, st.X, rtol=1e-9, atol=1e-9)
        assert np.allclose(yd, st.y, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_feasible_converges_and_is_certified(seed):
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], seed)
    prob, status, st = _solve(A, w["d_p"], w["d1"])
    assert status == ipm.OK and st.it <= 40
    sc = st.history[-1]
    # weak duality: a^T y - tr(CX) = tr(ZX) once the residuals vanish
    assert abs((sc["psi"] - sc["phi"]) - sc["trZX"]) < 1e-8 * (1 + abs(sc["psi"]))
    cert = certify.certify(prob, st.y)
    assert cert["verdict"] == 1
    # necessity: a certificate implies every vertex A(e_i) is Hurwitz and the
    # Lyapunov inequalities hold on a dense simplex grid (Thm 1)
    for Ai in A:
        assert np.linalg.eigvals(Ai).real.max() < 0
    assert certify.grid_check(prob, st.y, 20)["ok"]


def test_tiny_unstable_is_not_certified():
    w = synth.WORKLOADS["tiny_unstable"]
    for seed in (0, 1, 2):
        A = synth.system(w["n"], w["l"], w["s"], seed)
        # the grid falsifier finds an unstable alpha on these seeds
        assert certify.grid_max_real_eig(A, 1, w["l"], 50) >= 0
        prob, status, st = _solve(A, w["d_p"], w["d1"])
        assert status in (ipm.UNBOUNDED, ipm.MAXITER)
        assert certify.certify(prob, st.y)["verdict"] == 0


@pytest.mark.parametrize("signs,d_p,d1", [((-1, -2, -0.5), 1, 1), ((-1, 0.3, -2), 1, 1), ((-0.2, -0.1), 2, 2),
                                          ((0.4, -1), 1, 2), ((-3, -1, -1, -0.1), 2, 1)])
def test_scalar_systems(signs, d_p, d1):
    """n = 1: x' = (sum a_i alpha_i) x is robustly stable iff every a_i < 0, and
    then P(alpha) = p (sum alpha)^{d_p} is a certificate for any degrees."""
    A = np.array(signs, dtype=np.float64).reshape(-1, 1, 1)
    prob, status, st = _solve(A, d_p, d1)
    verdict = certify.certify(prob, st.y)["verdict"]
    assert verdict == int(all(a < 0 for a in signs))


@pytest.mark.parametrize("seed,shift", [(0, 0.0), (1, 0.0), (2, 1.5), (3, 1.2)])
def test_single_parameter_is_lyapunov(seed, shift):
    """l = 1: the LMIs reduce to P > 0, A^T P + P A < 0 (Lyapunov); certified iff
    A is Hurwitz, and then the textbook Lyapunov solution is a valid P too."""
    A = synth.system(4, 1, 0.0, seed) + shift * np.eye(4)
    hurwitz = np.linalg.eigvals(A[0]).real.max() < 0
    prob, status, st = _solve(A, 1, 1)
    cert = certify.certify(prob, st.y)
    assert cert["verdict"] == int(hurwitz)
    if hurwitz:
        Pl = scipy.linalg.solve_continuous_lyapunov(A[0].T, -np.eye(4))
        assert np.linalg.eigvalsh(Pl).min() > 0
        # our P satisfies the same strict inequalities
        P = prob.P_from_y(st.y)[0]
        assert np.linalg.eigvalsh(P).min() > 0
        assert np.linalg.eigvalsh(A[0].T @ P + P @ A[0]).max() < 0


def test_literal_and_structured_iterations_agree():
    prob = sdp.Problem(synth.system(3, 2, 0.3, 4), 1, 1)
    s1, s2 = ipm.start_point(prob), ipm.start_point(prob)
    for _ in range(5):
        ipm.newton_step(prob, s1, ipm.Options(schur="literal"))
        ipm.newton_step(prob, s2, ipm.Options(schur="structured"))
    assert np.allclose(s1.y, s2.y, rtol=1e-9, atol=1e-10)


def test_certificate_catches_wrong_sign():
    """Negating y (a sign slip) must destroy the certificate."""
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    prob, status, st = _solve(A, w["d_p"], w["d1"])
    assert certify.certify(prob, st.y)["verdict"] == 1
    assert certify.certify(prob, -st.y)["verdict"] == 0
