"""The large workload (n=100, l=3, d_p=2, d1=d2=4: K=30300, 64 blocks of
100x100) at full size, on outputs the oracle can compute one by one: the
Polya tables bit-exact, sampled columns of the FP64 Schur complement at a
random interior iterate against the definition Omega e_j = B(Z^{-1} B^T(e_j) X)
(Sec. IV-A), and the mixed-precision solve's certificate re-checked by the
oracle's eigenvalue test on the P_h it returns (Thm 1-2)."""

import numpy as np
import pytest

from oracle import certify, sdp
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


@pytest.fixture(scope="module")
def large():
    w = synth.WORKLOADS["large"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    return w, A, sdp.Problem(A, w["d_p"], w["d1"])


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_large_tables_bit_exact(bd, large):
    w, A, prob = large
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A, bd.psdp_default_opts())
    try:
        assert bd.psdp_sizes(h)["K"] == 30300 == prob.K
        beta, c = bd.psdp_get_tables(h)
        assert np.array_equal(beta, prob.beta) and np.array_equal(c, prob.c)
    finally:
        bd.psdp_destroy(h)


def test_large_schur_columns_match_oracle(bd, large):
    w, A, prob = large
    n, nb = w["n"], prob.nblk
    rng = np.random.default_rng(5)
    G = rng.normal(size=(nb, n, n))
    X = np.einsum("gij,gkj->gik", G, G) / n + np.eye(n)
    G = rng.normal(size=(nb, n, n))
    Z = np.einsum("gij,gkj->gik", G, G) / n + np.eye(n)
    cols = np.array([0, 5049, 5050, 30299], dtype=np.int32)   # ends of the first two block rows, the last column
    h = bd.psdp_setup(n, w["l"], w["d_p"], w["d1"], A, bd.psdp_default_opts())
    try:
        bd.psdp_load_iterate(h, X, Z, np.zeros(prob.K))
        got = bd.psdp_get_schur_cols(h, cols)
    finally:
        bd.psdp_destroy(h)
    Y = np.linalg.inv(Z)
    for q, j in enumerate(cols):
        e = np.zeros(prob.K)
        e[j] = 1.0
        ref = prob.schur_matvec(Y, X, e)
        assert _rel(got[q], ref) <= 1e-10, j


def test_large_mixed_solve_certified_by_oracle(bd, large):
    w, A, prob = large
    with bd.Solver(A, w["d_p"], w["d1"], precision=1) as s:
        status, iters, info = s.solve()
        verdict, _, _ = s.certify()
        y = bd.psdp_get_y(s.h)
    assert status == "OK" and verdict == 1
    assert info["relgap"] <= 1e-7
    assert certify.certify(prob, y)["verdict"] == 1
