"""Example 2 of Sec. V (the paper's only printed system data) through the oracle.

The six 3x3 coefficients are the paper's (tests/golden/example2_A.txt).  The
uncertainty set S_L = {a: a1 + a2 + a3 = 2L + 1, L <= a_i <= 1} is the image of
the simplex under a_i = (1 - L) alpha_i + L (alpha_1 + alpha_2 + alpha_3), and
the paper gives L_opt = -0.111 for min L such that the system is stable on S_L.

Pins: the transcription and the map reproduce that threshold by brute force
(eigenvalues on an alpha lattice, no SDP); the linear substitution matches
direct evaluation; the oracle's bisection bound never certifies below L_opt,
its certificate passes the independent alpha-grid check, and the bound does
not increase with the Polya exponent (Thm 2: a higher exponent keeps every
coefficient positive).
"""

import os

import numpy as np
import pytest

from oracle import certify, ipm, polya, sdp

L_OPT = -0.111


def load_example2():
    mats, cur = {}, None
    path = os.path.join(os.path.dirname(__file__), "golden", "example2_A.txt")
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("A"):
                cur = tuple(int(x) for x in line.split()[1:])
                mats[cur] = []
            else:
                mats[cur].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


def g_matrix(L):
    return (1.0 - L) * np.eye(3) + L * np.ones((3, 3))


def eval_poly(terms, b):
    return sum(c * np.prod([b[i] ** e[i] for i in range(len(b))]) for e, c in terms.items())


def max_real_eig_on_set(terms, L, N=60):
    worst = -np.inf
    for i in range(N + 1):
        for j in range(N + 1 - i):
            a = np.array([i, j, N - i - j]) / N
            worst = max(worst, np.linalg.eigvals(eval_poly(terms, g_matrix(L) @ a)).real.max())
    return worst


def coeffs_on_simplex(L):
    sub = polya.substitute_linear(load_example2(), g_matrix(L))
    return np.array([sub.get(tuple(m), np.zeros((3, 3))) for m in polya.monomials(3, 3)])


def certified(L, d_p, d1):
    prob = sdp.Problem(coeffs_on_simplex(L), d_p, d1, d_a=3)
    _, st = ipm.solve(prob, ipm.Options(eps=1e-8))
    return certify.certify(prob, st.y)["verdict"] == 1, prob, st


def oracle_bisect(d_p, d1, lo=-0.2, hi=1.0, iters=10, trace=None):
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        v = certified(mid, d_p, d1)[0]
        if trace is not None:
            trace.append((mid, int(v)))
        if v:
            hi = mid
        else:
            lo = mid
    return hi


def certificate_margin(L, d_p, d1, eps):
    """Signed margin of the certificate (reading R-A5) at scale L after an oracle
    solve to tolerance eps: min over every coefficient matrix M of
    lambda_min(M) - tau_c(M); certified exactly when it is positive."""
    prob = sdp.Problem(coeffs_on_simplex(L), d_p, d1, d_a=3)
    _, st = ipm.solve(prob, ipm.Options(eps=eps))
    coefP, coefL = certify.coefficient_matrices(prob, st.y)
    return min(float(np.linalg.eigvalsh(M).min()) - certify.tau_c(M) for M in list(coefP) + list(coefL))


def verdict_is_determined(L, d_p, d1, eps=1e-8, factor=4.0):
    """(determined, verdict) at scale L.  The stopping rule accepts any iterate
    whose gap and residuals are below eps, and at a certified scale near the
    threshold the margin of the final iterate shrinks with the iterate's distance
    to the optimum (the optimal dual has a singular Lyapunov coefficient), so two
    correct solvers can stop on iterates of different verdicts.  The change of the
    margin when the stopping tolerance moves by one decade (10 eps to eps) measures
    that dependence; the verdict is determined when the margin at eps exceeds
    `factor` times it."""
    m = certificate_margin(L, d_p, d1, eps)
    m_loose = certificate_margin(L, d_p, d1, 10.0 * eps)
    return abs(m) > factor * abs(m - m_loose), int(m > 0)


def determined_many(points, processes=None):
    """verdict_is_determined for many (L, d_p, d1) in a process pool started
    with spawn (safe next to a process that already uses a GPU)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    points = list(points)
    if not points:
        return []
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        workers = processes or max(1, min(len(points), os.cpu_count() or 1, 16))
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_determined_star, points))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _determined_star(args):
    return verdict_is_determined(*args)


def test_transcription_reproduces_the_printed_threshold():
    terms = load_example2()
    assert len(terms) == 6 and all(sum(e) == 3 for e in terms)
    assert max_real_eig_on_set(terms, L_OPT + 0.002) < 0.0      # stable just above L_opt
    assert max_real_eig_on_set(terms, L_OPT - 0.003) > 0.0      # unstable just below


def test_substitution_matches_direct_evaluation():
    rng = np.random.default_rng(0)
    terms = {m: rng.normal(size=(2, 2)) for m in polya.monomials(3, 3)}
    M = rng.normal(size=(3, 3))
    sub = polya.substitute_linear(terms, M)
    assert all(sum(e) == 3 for e in sub)
    for _ in range(5):
        a = rng.random(3)
        assert np.allclose(eval_poly(sub, a), eval_poly(terms, M @ a), rtol=1e-12, atol=1e-12)
    ident = polya.substitute_linear(terms, np.eye(3))
    assert all(np.array_equal(ident[e], terms[e]) for e in terms)


def test_oracle_bound_is_sound_and_certificate_checks_on_grid():
    b11 = oracle_bisect(1, 1)
    assert L_OPT < b11 < 1.0
    ok, prob, st = certified(b11, 1, 1)
    assert ok
    chk = certify.grid_check(prob, st.y, 12)
    assert chk["ok"] and chk["minP"] > 0 and chk["maxQ"] < 0


@pytest.mark.slow
def test_oracle_bound_does_not_grow_with_the_polya_exponent():
    assert oracle_bisect(1, 2) <= oracle_bisect(1, 1) + 1e-12
