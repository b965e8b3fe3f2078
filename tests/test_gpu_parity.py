"""GPU parity: the sm_103a library through its C ABI against the FP64 CPU oracle.

Tolerances: integer tables bit-exact; the operators B^T, B and the Schur
complement within 1e-12 / 1e-10 relative (FP64 with different summation order
only); one Newton step from the same iterate within 1e-8 relative (the step
solves Omega dy = r, whose conditioning amplifies rounding by kappa(Omega));
verdicts identical; the optimal dual objective (unique although the optimal P
is not) within 1e-6 relative at eps = 1e-8.
"""

import numpy as np
import pytest

from oracle import certify, ipm, polya, sdp
from paper_1411_3769_gb300 import synth

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


def _spd(rng, nb, n):
    G = rng.normal(size=(nb, n, n))
    return np.einsum("gij,gkj->gik", G, G) / n + np.eye(n)


TABLE_CASES = [dict(n=3, l=2, d_p=1, d1=1), dict(n=3, l=4, d_p=2, d1=3), dict(n=2, l=3, d_p=2, d1=4),
               dict(n=2, l=3, d_p=0, d1=2), dict(n=2, l=2, d_p=1, d1=0), dict(n=2, l=3, d_p=1, d1=2, d2=3),
               dict(n=2, l=2, d_p=2, d1=1, d_a=3), dict(n=2, l=8, d_p=1, d1=1), dict(n=2, l=1, d_p=3, d1=2)]


@pytest.mark.parametrize("cs", TABLE_CASES)
def test_tables_bit_exact(bd, cs):
    cs = dict(cs)
    d_a = cs.pop("d_a", 1)
    d2 = cs.pop("d2", None)
    n, l = cs["n"], cs["l"]
    rng = np.random.default_rng(0)
    A = rng.normal(size=(polya.f_card(l, d_a), n, n))
    opts = bd.psdp_default_opts(d_a=d_a, d2=-1 if d2 is None else d2)
    h = bd.psdp_setup(n, l, cs["d_p"], cs["d1"], A, opts)
    try:
        beta, c = bd.psdp_get_tables(h)
        prob = sdp.Problem(A, cs["d_p"], cs["d1"], d2=d2, d_a=d_a)
        assert beta.dtype == np.int32 and np.array_equal(beta, prob.beta)
        assert np.array_equal(c, prob.c)
    finally:
        bd.psdp_destroy(h)


@pytest.mark.parametrize("cs", [dict(n=5, l=2, d_p=1, d1=1), dict(n=7, l=3, d_p=2, d1=2), dict(n=4, l=2, d_p=2, d1=1, d_a=2),
                                dict(n=20, l=4, d_p=2, d1=3), dict(n=33, l=2, d_p=1, d1=1),
                                # exact-tile block products: n = 40 (20 x 20 tiles), 50 (25 x 25)
                                dict(n=40, l=2, d_p=1, d1=1), dict(n=50, l=3, d_p=1, d1=1)])
def test_operators_match_oracle(bd, cs):
    cs = dict(cs)
    d_a = cs.pop("d_a", 1)
    n, l = cs["n"], cs["l"]
    rng = np.random.default_rng(1)
    A = rng.normal(size=(polya.f_card(l, d_a), n, n)) / np.sqrt(n)
    prob = sdp.Problem(A, cs["d_p"], cs["d1"], d_a=d_a)
    h = bd.psdp_setup(n, l, cs["d_p"], cs["d1"], A, bd.psdp_default_opts(d_a=d_a))
    try:
        v = rng.normal(size=prob.K)
        assert _rel(bd.psdp_apply_BT(h, v), prob.BT(v)) <= 1e-12
        W = rng.normal(size=(prob.nblk, n, n))
        assert _rel(bd.psdp_apply_B(h, W), prob.Bop(W)) <= 1e-12
    finally:
        bd.psdp_destroy(h)


SCHUR_CASES = [dict(n=5, l=2, d_p=1, d1=1), dict(n=6, l=3, d_p=2, d1=2), dict(n=9, l=2, d_p=1, d1=3),
               dict(n=20, l=4, d_p=2, d1=3), dict(n=13, l=3, d_p=0, d1=2), dict(n=3, l=2, d_p=2, d1=1, d_a=2),
               dict(n=1, l=3, d_p=1, d1=1), dict(n=70, l=1, d_p=0, d1=0), dict(n=40, l=2, d_p=1, d1=1)]


@pytest.mark.parametrize("cs", SCHUR_CASES)
def test_schur_matches_oracle(bd, cs):
    cs = dict(cs)
    d_a = cs.pop("d_a", 1)
    n, l = cs["n"], cs["l"]
    rng = np.random.default_rng(2)
    A = rng.normal(size=(polya.f_card(l, d_a), n, n)) / np.sqrt(n)
    prob = sdp.Problem(A, cs["d_p"], cs["d1"], d_a=d_a)
    h = bd.psdp_setup(n, l, cs["d_p"], cs["d1"], A, bd.psdp_default_opts(d_a=d_a))
    try:
        # cold start X = Z = I
        I = prob.identity_blocks()
        Om = bd.psdp_get_schur(h)
        assert _rel(Om, prob.schur_structured(I, I)) <= 1e-10
        # a random interior iterate
        X, Z = _spd(rng, prob.nblk, n), _spd(rng, prob.nblk, n)
        y = rng.normal(size=prob.K)
        bd.psdp_load_iterate(h, X, Z, y)
        Om = bd.psdp_get_schur(h)
        ref = prob.schur_structured(np.linalg.inv(Z), X)
        assert _rel(Om, ref) <= 1e-10
        if prob.K <= 400:
            assert _rel(Om, prob.schur_literal(np.linalg.inv(Z), X)) <= 1e-10
    finally:
        bd.psdp_destroy(h)


@pytest.mark.parametrize("name,seed,k", [("tiny", 0, 3), ("tiny", 1, 8), ("tiny_unstable", 0, 5)])
def test_newton_step_matches_oracle(bd, name, seed, k):
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], seed)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    st = ipm.start_point(prob)
    for _ in range(k):
        ipm.newton_step(prob, st, ipm.Options())
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        bd.psdp_load_iterate(h, st.X, st.Z, st.y)
        info_o = ipm.newton_step(prob, st, ipm.Options())
        s, info = bd.psdp_step(h)
        assert s == 0
        X, Z, y = bd.psdp_get_iterate(h)
        assert abs(info[6] - info_o["tp"]) <= 1e-8 and abs(info[7] - info_o["td"]) <= 1e-8
        assert _rel(y, st.y) <= 1e-8
        assert _rel(X, st.X) <= 1e-8
        assert _rel(Z, st.Z) <= 1e-8
        sc = ipm.scalars(prob, st)
        assert abs(info[0] - sc["phi"]) <= 1e-8 * (1 + abs(sc["phi"]))
        assert abs(info[1] - sc["psi"]) <= 1e-8 * (1 + abs(sc["psi"]))
    finally:
        bd.psdp_destroy(h)


@pytest.mark.parametrize("name,seed", [("tiny", 0), ("tiny", 1), ("tiny", 2), ("tiny_unstable", 0),
                                       ("tiny_unstable", 1), ("tiny_unstable", 2)])
def test_tiny_solve_verdicts(bd, name, seed):
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], seed)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    st_o, state = ipm.solve(prob)
    cert_o = certify.certify(prob, state.y)
    with bd.Solver(A, w["d_p"], w["d1"]) as s:
        status, iters, info = s.solve()
        verdict, minP, maxL = s.certify()
        y = bd.psdp_get_y(s.h)
        # the GPU certificate on the GPU's own y agrees with the oracle's certificate of that y
        cert_y = certify.certify(prob, y)
        assert verdict == cert_y["verdict"]
        assert abs(minP - cert_y["minP_margin"]) <= 1e-9 * (1 + abs(cert_y["minP_margin"]))
        assert abs(maxL - cert_y["maxLyap_margin"]) <= 1e-9 * (1 + abs(cert_y["maxLyap_margin"]))
    assert verdict == cert_o["verdict"]
    assert status.removeprefix("E") == st_o
    if status == "OK":
        assert info["relgap"] <= 1e-7 and abs(iters - state.it) <= 2


def test_mid_config_solve(bd):
    """n=20, l=4, d_p=2, d1=3 (K=2100, 140 blocks), s=0.3, gap 1e-8."""
    w = synth.WORKLOADS["mid"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    st_o, state = ipm.solve(prob, ipm.Options(eps=1e-8))
    cert_o = certify.certify(prob, state.y)
    with bd.Solver(A, w["d_p"], w["d1"], eps=1e-8) as s:
        status, iters, info = s.solve()
        verdict, minP, maxL = s.certify()
    assert status == st_o == "OK"
    assert verdict == cert_o["verdict"] == 1
    psi_o = state.history[-1]["psi"]
    assert abs(info["psi"] - psi_o) <= 1e-6 * abs(psi_o)
    assert abs(iters - state.it) <= 3


def test_grid_check_matches_oracle(bd):
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    with bd.Solver(A, w["d_p"], w["d1"]) as s:
        s.solve()
        y = bd.psdp_get_y(s.h)
        mp, mq = bd.psdp_grid_check(s.h, 30)
    g = certify.grid_check(prob, y, 30)
    assert abs(mp - g["minP"]) <= 1e-10 * (1 + abs(g["minP"]))
    assert abs(mq - g["maxQ"]) <= 1e-10 * (1 + abs(g["maxQ"]))
    assert g["ok"] and mp > 0 and mq < 0


@pytest.mark.parametrize("signs,d_p,d1", [((-1.0, -2.0, -0.5), 1, 1), ((-1.0, 0.3, -2.0), 1, 1), ((-0.2, -0.1), 2, 2)])
def test_scalar_systems(bd, signs, d_p, d1):
    A = np.array(signs).reshape(-1, 1, 1)
    with bd.Solver(A, d_p, d1) as s:
        s.solve()
        verdict = s.certify()[0]
    assert verdict == int(all(a < 0 for a in signs))


@pytest.mark.parametrize("seed,shift", [(0, 0.0), (2, 1.5)])
def test_single_parameter(bd, seed, shift):
    A = synth.system(4, 1, 0.0, seed) + shift * np.eye(4)
    hurwitz = np.linalg.eigvals(A[0]).real.max() < 0
    with bd.Solver(A, 1, 1) as s:
        s.solve()
        assert s.certify()[0] == int(hurwitz)


def test_non_pd_block_is_reported_and_iterate_kept(bd):
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        X, Z, y = bd.psdp_get_iterate(h)
        Z[3] = -np.eye(w["n"])
        bd.psdp_load_iterate(h, X, Z, y)
        s, _ = bd.psdp_step(h)
        assert bd.STATUS[s] in ("ECHOL_BLOCK", "ECHOL_SCHUR")
        X2, Z2, y2 = bd.psdp_get_iterate(h)
        assert np.array_equal(X2, X) and np.array_equal(Z2, Z) and np.array_equal(y2, y)
        # the context stays usable
        X[:], Z[:] = np.eye(w["n"]), np.eye(w["n"])
        bd.psdp_load_iterate(h, X, Z, np.zeros_like(y))
        assert bd.psdp_step(h)[0] == 0
    finally:
        bd.psdp_destroy(h)


def test_graph_and_eager_agree(bd):
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 1)
    ys = []
    for g in (0, 1):
        with bd.Solver(A, w["d_p"], w["d1"], use_graph=g) as s:
            for _ in range(6):
                s.step()
            ys.append(bd.psdp_get_y(s.h))
    assert np.array_equal(ys[0], ys[1])
