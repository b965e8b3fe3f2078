"""The generalised inequality (Sec. III-C, Eq. LMI_general with one term,
A~ = A(alpha)^T, B~ = I) on the GPU: A(alpha)^T P(alpha) + P(alpha) A(alpha) + R(alpha) < 0
with a caller-chosen dual objective a, through psdp_set_constant_term and
psdp_set_objective, against the oracle.

Tolerances as in the other parity tests: one Newton step from the same iterate
to 1e-8 relative; the optimal value a^T y* (unique) to 1e-6 relative of the
oracle's and of the H2 closed form (tr(B^T W_o B), scipy's Lyapunov solver);
certificate margins to 1e-9 of the oracle's certificate of the same y.
"""

import numpy as np
import pytest

from oracle import certify, ipm, sdp
from paper_1411_3769_gb300 import synth
from tests.test_oracle_general import h2_squared, svec_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_3769_gb300 import build
    build.build()
    from paper_1411_3769_gb300 import binding
    binding._lib()
    return binding


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _problem(n, l, d_p, d1, s, seed, d_r):
    rng = np.random.default_rng(seed + 100)
    A = synth.system(n, l, s, seed)
    from oracle import polya
    Nr = polya.f_card(l, d_r)
    G = rng.normal(size=(Nr, n, n)) / np.sqrt(n)
    R = 0.05 * np.einsum("rij,rkj->rik", G, G)       # positive semidefinite coefficients
    K = polya.f_card(l, d_p) * n * (n + 1) // 2
    a = rng.uniform(0.5, 1.5, size=K)
    return A, R, a


@pytest.mark.parametrize("n,l,d_p,d1,d_r,k", [(5, 2, 1, 1, 1, 3), (4, 3, 2, 1, 0, 5), (20, 4, 2, 3, 2, 4)])
def test_newton_step_with_constant_term_and_objective(bd, n, l, d_p, d1, d_r, k):
    A, R, a = _problem(n, l, d_p, d1, 0.3, 1, d_r)
    prob = sdp.Problem(A, d_p, d1, R=R, d_r=d_r, a=a)
    st = ipm.start_point(prob)
    for _ in range(k):
        assert ipm.newton_step(prob, st, ipm.Options())["status"] == ipm.OK
    h = bd.psdp_setup(n, l, d_p, d1, A)
    try:
        bd.psdp_set_constant_term(h, d_r, R)
        bd.psdp_set_objective(h, a)
        bd.psdp_load_iterate(h, st.X, st.Z, st.y)
        info_o = ipm.newton_step(prob, st, ipm.Options())
        s, info = bd.psdp_step(h)
        assert s == 0
        X, Z, y = bd.psdp_get_iterate(h)
        assert abs(info[6] - info_o["tp"]) <= 1e-8 and abs(info[7] - info_o["td"]) <= 1e-8
        assert _rel(y, st.y) <= 1e-8 and _rel(X, st.X) <= 1e-8 and _rel(Z, st.Z) <= 1e-8
        sc = ipm.scalars(prob, st)
        for i, key in ((0, "phi"), (1, "psi"), (3, "pres"), (4, "dres")):
            assert abs(info[i] - sc[key]) <= 1e-8 * (1 + abs(sc[key])), key
    finally:
        bd.psdp_destroy(h)


@pytest.mark.parametrize("seed", [0, 1])
def test_h2_norm_on_the_gpu(bd, seed):
    rng = np.random.default_rng(seed)
    A = synth.system(4, 1, 0.0, seed)[0]
    B, Cz = rng.normal(size=(4, 2)), rng.normal(size=(2, 4))
    h2, _ = h2_squared(A, B, Cz)
    a = svec_weights(B @ B.T)
    with bd.Solver(A[None], 1, 0, delta=1e-9, eps=1e-9) as s:
        bd.psdp_set_constant_term(s.h, 0, (Cz.T @ Cz)[None])
        bd.psdp_set_objective(s.h, a)
        status, iters, info = s.solve()
        verdict = s.certify()[0]
    assert status == "OK" and verdict == 1
    assert abs(info["psi"] - h2) <= 1e-6 * h2


def test_robust_h2_bound_matches_oracle(bd):
    n, l = 6, 2
    rng = np.random.default_rng(3)
    A = synth.system(n, l, 0.3, 3)
    Bm, Cz = rng.normal(size=(n, 2)), rng.normal(size=(1, n))
    R = (Cz.T @ Cz)[None]
    a = np.concatenate([svec_weights(Bm @ Bm.T)] * 2)
    prob = sdp.Problem(A, 1, 1, delta=1e-9, R=R, d_r=0, a=a)
    st_o, state = ipm.solve(prob, ipm.Options(eps=1e-9))
    psi_o = float(prob.a @ state.y)
    with bd.Solver(A, 1, 1, delta=1e-9, eps=1e-9) as s:
        bd.psdp_set_constant_term(s.h, 0, R)
        bd.psdp_set_objective(s.h, a)
        status, iters, info = s.solve()
        verdict, minP, maxL = s.certify()
        y = bd.psdp_get_y(s.h)
        mp, mq = bd.psdp_grid_check(s.h, 12)
    assert status == st_o == "OK"
    assert abs(info["psi"] - psi_o) <= 1e-6 * abs(psi_o)
    cert = certify.certify(prob, y)
    assert verdict == cert["verdict"] == 1
    assert abs(minP - cert["minP_margin"]) <= 1e-9 * (1 + abs(cert["minP_margin"]))
    assert abs(maxL - cert["maxLyap_margin"]) <= 1e-9 * (1 + abs(cert["maxLyap_margin"]))
    g = certify.grid_check(prob, y, 12)
    assert abs(mp - g["minP"]) <= 1e-10 * (1 + abs(g["minP"]))
    assert abs(mq - g["maxQ"]) <= 1e-10 * (1 + abs(g["maxQ"]))
    assert g["ok"] and mq < 0


def test_generalised_form_arguments_are_checked(bd):
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        R = np.zeros((1, w["n"], w["n"]))
        R[0, 0, 1] = 1.0                                 # not symmetric
        with pytest.raises(bd.PsdpError):
            bd.psdp_set_constant_term(h, 0, R)
        with pytest.raises(bd.PsdpError):               # degree above d_p + d_a + d2 = 3
            bd.psdp_set_constant_term(h, 4, np.zeros((5, w["n"], w["n"])))
        a = np.ones(bd.psdp_sizes(h)["K"])
        a[3] = np.nan
        with pytest.raises(bd.PsdpError):
            bd.psdp_set_objective(h, a)
        # R = 0 and a = 1 give back the plain problem, bit for bit
        bd.psdp_set_constant_term(h, 0, np.zeros((1, w["n"], w["n"])))
        bd.psdp_set_objective(h, np.ones(bd.psdp_sizes(h)["K"]))
        s1 = [bd.psdp_step(h)[1] for _ in range(3)]
    finally:
        bd.psdp_destroy(h)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        s0 = [bd.psdp_step(h)[1] for _ in range(3)]
    finally:
        bd.psdp_destroy(h)
    assert np.array_equal(np.array(s0)[:, :12], np.array(s1)[:, :12])
