"""Mixed-precision path (3xTF32 tensor-core Schur complement and Cholesky, FP64
PCG refinement) against the FP64 oracle.

Stated errors: the FP32 Schur complement is within 1e-5 of max|Omega| (operands
rounded to FP32, 3xTF32 products ~2^-21 relative, FP32 accumulation over the
contraction); the Newton directions are refined in FP64 until the relative
residual is 1e-12, so a mixed step from the same iterate matches the FP64 step
to 1e-8; a full mixed solve reaches the same verdict and the same optimal dual
objective (within 1e-6 relative) as the FP64 oracle.
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
    return float(np.abs(np.asarray(a, np.float64) - b).max() / np.abs(b).max())


@pytest.mark.parametrize("cs", [dict(n=5, l=2, d_p=1, d1=1), dict(n=20, l=4, d_p=2, d1=3),
                                dict(n=9, l=3, d_p=2, d1=2), dict(n=33, l=2, d_p=1, d1=1)])
def test_mixed_schur(bd, cs):
    n, l = cs["n"], cs["l"]
    rng = np.random.default_rng(5)
    A = rng.normal(size=(l, n, n)) / np.sqrt(n)
    prob = sdp.Problem(A, cs["d_p"], cs["d1"])
    h = bd.psdp_setup(n, l, cs["d_p"], cs["d1"], A, bd.psdp_default_opts(precision=1))
    try:
        I = prob.identity_blocks()
        assert _rel(bd.psdp_get_schur_mixed(h), prob.schur_structured(I, I)) <= 1e-5
        G = rng.normal(size=(prob.nblk, n, n))
        X = np.einsum("gij,gkj->gik", G, G) / n + np.eye(n)
        G = rng.normal(size=(prob.nblk, n, n))
        Z = np.einsum("gij,gkj->gik", G, G) / n + np.eye(n)
        bd.psdp_load_iterate(h, X, Z, rng.normal(size=prob.K))
        ref = prob.schur_structured(np.linalg.inv(Z), X)
        assert _rel(bd.psdp_get_schur_mixed(h), ref) <= 1e-5
    finally:
        bd.psdp_destroy(h)


@pytest.mark.parametrize("name,seed,k", [("tiny", 0, 4), ("mid", 0, 12)])
def test_mixed_step_matches_oracle(bd, name, seed, k):
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], seed)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    st = ipm.start_point(prob)
    for _ in range(k):
        ipm.newton_step(prob, st, ipm.Options())
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A, bd.psdp_default_opts(precision=1))
    try:
        bd.psdp_load_iterate(h, st.X, st.Z, st.y)
        ipm.newton_step(prob, st, ipm.Options())
        s, info = bd.psdp_step(h)
        assert s == 0 and info[13] == 0.0          # no fallback to FP64
        # a sound FP32 factor preconditions both systems to the 1e-12 target in a
        # few iterations each (8 is the cap per solve)
        assert info[12] <= 10
        X, Z, y = bd.psdp_get_iterate(h)
        assert np.abs(y - st.y).max() <= 1e-8 * (1 + np.abs(st.y).max())
        assert np.abs(X - st.X).max() <= 1e-8 * (1 + np.abs(st.X).max())
    finally:
        bd.psdp_destroy(h)


@pytest.mark.parametrize("name,seed", [("tiny", 0), ("tiny_unstable", 0), ("mid", 0)])
def test_mixed_solve_verdict(bd, name, seed):
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], seed)
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    eps = 1e-7
    st_o, state = ipm.solve(prob, ipm.Options(eps=eps))
    cert_o = certify.certify(prob, state.y)
    with bd.Solver(A, w["d_p"], w["d1"], precision=1, eps=eps) as s:
        status, iters, info = s.solve()
        verdict, minP, maxL = s.certify()
    assert verdict == cert_o["verdict"]
    assert status.removeprefix("E") == st_o
    if st_o == "OK":
        psi_o = state.history[-1]["psi"]
        assert abs(info["psi"] - psi_o) <= 1e-6 * abs(psi_o)
        assert abs(iters - state.it) <= 3
