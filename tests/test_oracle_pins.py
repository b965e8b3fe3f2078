"""Pins of oracle functions that the first tests left unpinned.

* grid_check (Thm 1 on the simplex lattice): closed forms that a transposed
  Lyapunov form or a wrong exponent order would miss, and the Lyapunov theorem
  at a lattice point where A(alpha) is not Hurwitz.
* max_step (reading R-A9, the exact largest step of Sec. IV-A's line search):
  brute-force bisection on lambda_min(X + t D) >= 0.
* adam: three steps with varying gradients against values worked out by hand,
  and the constant-gradient invariant that holds at every t.
"""

import math

import numpy as np
import pytest

from oracle import certify, ipm, mlp, sdp
from paper_1411_3769_gb300 import synth


# ------------------------------------------------------------------ grid_check
def test_grid_check_scalar_case_is_the_scalar_polynomial():
    """n = 1, l = 2, d_p = 2: P(alpha) = p20 a1^2 + p11 a1 a2 + p02 a2^2 and
    A(alpha) = a1 x1 + a2 x2, so Q = 2 A P; over the lattice alpha = (i/N, 1 - i/N)
    the extremes are those of two scalar polynomials.  The values are chosen
    asymmetric, so evaluating P with the exponent order reversed changes maxQ."""
    a = np.array([-1.0, 0.3])
    p = np.array([2.0, -0.5, 0.05])          # coefficients of (2,0), (1,1), (0,2)
    prob = sdp.Problem(a.reshape(2, 1, 1), 2, 1)
    N = 16
    res = certify.grid_check(prob, p, N)
    Pvals, Qvals, Qswap = [], [], []
    for i in range(N + 1):
        x1, x2 = i / N, 1 - i / N
        Pa = p[0] * x1 * x1 + p[1] * x1 * x2 + p[2] * x2 * x2
        Pr = p[2] * x1 * x1 + p[1] * x1 * x2 + p[0] * x2 * x2
        Aa = a[0] * x1 + a[1] * x2
        Pvals.append(Pa)
        Qvals.append(2 * Aa * Pa)
        Qswap.append(2 * Aa * Pr)
    assert abs(max(Qvals) - max(Qswap)) > 1e-2        # the case separates the two orders
    assert res["minP"] == pytest.approx(min(Pvals), rel=1e-14, abs=1e-15)
    assert res["maxQ"] == pytest.approx(max(Qvals), rel=1e-14, abs=1e-15)
    assert res["ok"] == (min(Pvals) > 0 and max(Qvals) < 0)


def test_grid_check_uses_the_transpose_on_the_left():
    """l = 1, A = [[-1, 1], [0, -1]], P = diag(1, p): A^T P + P A = [[-2, 1], [1, -2p]]
    has largest eigenvalue -(1 + p) + sqrt((1 - p)^2 + 1) > 0 at p = 0.01, while
    the transposed form A P + P A^T = [[-2, p], [p, -2p]] is negative definite."""
    pv = 0.01
    A = np.array([[[-1.0, 1.0], [0.0, -1.0]]])
    prob = sdp.Problem(A, 1, 1)
    y = np.array([1.0, pv, 0.0])              # svec: (0,0), (1,1), (0,1)
    res = certify.grid_check(prob, y, 3)
    lam = -(1 + pv) + math.sqrt((1 - pv) ** 2 + 1.0)
    lam_t = -(1 + pv) + math.sqrt((1 - pv) ** 2 + pv * pv)
    assert lam > 0.3 and lam_t < 0
    assert res["maxQ"] == pytest.approx(lam, rel=1e-13)
    assert res["minP"] == pytest.approx(pv, rel=1e-13)
    assert res["ok"] is False


def test_grid_check_rejects_any_P_where_A_is_not_hurwitz():
    """Lyapunov: P > 0 and A^T P + P A < 0 imply A Hurwitz.  On a system whose
    lattice has a point with max Re lambda(A(alpha)) >= 0, every P that is positive
    definite on the lattice (here the certificate of a stable system) must give
    maxQ >= 0 there, and the check must fail."""
    w = synth.WORKLOADS["tiny"]
    A_ok = synth.system(w["n"], w["l"], w["s"], 0)
    prob_ok = sdp.Problem(A_ok, w["d_p"], w["d1"])
    status, st = ipm.solve(prob_ok)
    assert status == ipm.OK and certify.certify(prob_ok, st.y)["verdict"] == 1
    wu = synth.WORKLOADS["tiny_unstable"]
    A_bad = synth.system(wu["n"], wu["l"], wu["s"], 0)
    N = 50
    assert certify.grid_max_real_eig(A_bad, 1, wu["l"], N) >= 0
    prob_bad = sdp.Problem(A_bad, w["d_p"], w["d1"])
    res = certify.grid_check(prob_bad, st.y, N)
    assert res["minP"] > 0
    assert res["maxQ"] >= 0 and res["ok"] is False
    # the point itself, checked by hand: P(alpha) = a1 P_1 + a2 P_2 (d_p = 1)
    P = prob_ok.P_from_y(st.y)
    worst = -np.inf
    for i in range(N + 1):
        al = (i / N, 1 - i / N)
        Aa = al[0] * A_bad[0] + al[1] * A_bad[1]
        if np.linalg.eigvals(Aa).real.max() >= 0:
            Pa = al[0] * P[0] + al[1] * P[1]
            worst = max(worst, np.linalg.eigvalsh(Aa.T @ Pa + Pa @ Aa).max())
    assert worst >= 0 and res["maxQ"] >= worst


# -------------------------------------------------------------------- max_step
def _bisect_step(X, D, iters=200):
    """sup{t >= 0: lambda_min(X_g + t D_g) >= 0 for every block}, by bisection."""
    def ok(t):
        return all(np.linalg.eigvalsh(Xb + t * Db).min() >= 0 for Xb, Db in zip(X, D))
    hi = 1.0
    while ok(hi):
        hi *= 2.0
        if hi > 1e12:
            return math.inf
    lo = 0.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo


def _spd(rng, n, cond):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return (Q * np.geomspace(1.0, 1.0 / cond, n)) @ Q.T


@pytest.mark.parametrize("seed", range(6))
def test_max_step_matches_bisection(seed):
    rng = np.random.default_rng(seed)
    n, nb = 6, 4
    X = np.stack([_spd(rng, n, 10.0 ** rng.uniform(0, 4)) for _ in range(nb)])
    D = rng.normal(size=(nb, n, n))
    D = 0.5 * (D + np.swapaxes(D, 1, 2)) * 10.0 ** rng.uniform(-2, 1)
    D[seed % nb] = _spd(rng, n, 5.0)        # one block with D >= 0 puts no limit
    t = ipm.max_step(X, D)
    tb = _bisect_step(X, D)
    assert math.isfinite(t)
    assert abs(t - tb) <= 1e-10 * tb


def test_max_step_is_infinite_when_every_direction_is_psd():
    rng = np.random.default_rng(11)
    X = np.stack([_spd(rng, 5, 100.0) for _ in range(3)])
    D = np.stack([_spd(rng, 5, 10.0) for _ in range(3)])
    D[1] = 0.0
    assert ipm.max_step(X, D) == math.inf
    assert _bisect_step(X, D) == math.inf


def test_max_step_closed_form_diagonal():
    """Diagonal blocks: the largest step is min over entries with d < 0 of x / (-d)."""
    X = np.array([np.diag([2.0, 1.0, 4.0]), np.diag([1.0, 3.0, 0.5])])
    D = np.array([np.diag([-1.0, 0.5, -8.0]), np.diag([0.0, -0.25, 1.0])])
    assert ipm.max_step(X, D) == pytest.approx(0.5, rel=1e-15)


# ------------------------------------------------------------------------ adam
def test_adam_three_steps_by_hand():
    """g = 1, 2, -1 with lr = 0.1, b1 = 0.9, b2 = 0.999, eps = 0.  By hand:
    t=1: m = 1/10, v = 1/1000, m^ = v^ = 1, step 0.1;
    t=2: m = 29/100, v = 4999/10^6, m^ = 29/19, v^ = 4999/1999;
    t=3: m = 161/1000, v = 5994001/10^9, m^ = 161/271, v^ = 5994001/2997001."""
    p = np.array([0.0])
    m, v = np.zeros(1), np.zeros(1)
    expect_m = [1 / 10, 29 / 100, 161 / 1000]
    expect_v = [1 / 1000, 4999 / 1e6, 5994001 / 1e9]
    expect_p = [-0.1,
                -0.1 - 0.1 * (29 / 19) / math.sqrt(4999 / 1999),
                -0.1 - 0.1 * (29 / 19) / math.sqrt(4999 / 1999) - 0.1 * (161 / 271) / math.sqrt(5994001 / 2997001)]
    for t, g in enumerate([1.0, 2.0, -1.0], start=1):
        mlp.adam(p, np.array([g]), m, v, t=t, lr=0.1, eps=0.0)
        assert m[0] == pytest.approx(expect_m[t - 1], rel=1e-14)
        assert v[0] == pytest.approx(expect_v[t - 1], rel=1e-13)
        assert p[0] == pytest.approx(expect_p[t - 1], rel=1e-14)
    assert p[0] == pytest.approx(-0.238527132939205, rel=1e-13)


def test_adam_constant_gradient_steps_are_lr_at_every_t():
    """With a constant gradient the bias-corrected moments are g and g^2 at every
    t, so each step moves by lr * g / (|g| + eps)."""
    g = np.array([0.5, -4.0, 3e-2])
    p = np.zeros(3)
    m, v = np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        before = p.copy()
        mlp.adam(p, g, m, v, t=t, lr=0.01)
        assert np.allclose(before - p, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
