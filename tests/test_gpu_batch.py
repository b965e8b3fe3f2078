"""Batched uneven instances (one batch graph per interior-point iteration) and
the step-configuration autotuner.

A batched instance runs the very same captured step graph as a single solve,
so its iterate, iteration count and status must be bit-identical to solving it
alone; verdicts must equal the oracle's.
"""

import os

import numpy as np
import pytest

from oracle import certify, ipm, sdp
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


def _instances(count, base):
    return synth.batch_instances(count, base_seed=base, n_range=(4, 10))


@pytest.mark.parametrize("precisions", [(0,), (0, 1)])
def test_batch_is_bit_identical_to_single_solves(bd, precisions):
    inst = _instances(10, 4000)
    handles = []
    try:
        for i, d in enumerate(inst):
            prec = precisions[i % len(precisions)]
            handles.append(bd.psdp_setup(d["n"], d["l"], d["d_p"], d["d1"], d["A"],
                                         bd.psdp_default_opts(precision=prec, max_iter=60)))
        status, iters = bd.psdp_solve_batch(handles)
        ys = [bd.psdp_get_y(h) for h in handles]
        verdicts = [bd.psdp_certify(h)[0] for h in handles]
    finally:
        for h in handles:
            bd.psdp_destroy(h)
    for i, d in enumerate(inst):
        prec = precisions[i % len(precisions)]
        with bd.Solver(d["A"], d["d_p"], d["d1"], precision=prec, max_iter=60) as s:
            st1, it1, _ = s.solve()
            y1 = bd.psdp_get_y(s.h)
            v1 = s.certify()[0]
        assert (status[i], iters[i]) == (st1, it1), i
        assert np.array_equal(ys[i], y1), i
        assert verdicts[i] == v1
        prob = sdp.Problem(d["A"], d["d_p"], d["d1"])
        st_o, state = ipm.solve(prob, ipm.Options(max_iter=60))
        assert verdicts[i] == certify.certify(prob, state.y)["verdict"], i


def test_autotune_choice_and_cache(bd, tmp_path):
    w = synth.WORKLOADS["mid"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    cache = os.path.join(tmp_path, "tune.txt")
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        X0, Z0, y0 = bd.psdp_get_iterate(h)
        choice, ms = bd.psdp_autotune(h, cache)
        assert choice in (0, 1, 2) and np.all(ms > 0) and ms[choice] == ms.min()
        X1, Z1, y1 = bd.psdp_get_iterate(h)          # the iterate is restored
        assert np.array_equal(X0, X1) and np.array_equal(y0, y1)
        status, iters, info = bd.psdp_solve(h)
        assert bd.STATUS[status] == "OK" and bd.psdp_certify(h)[0] == 1
    finally:
        bd.psdp_destroy(h)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        choice2, ms2 = bd.psdp_autotune(h, cache)     # answered from the cache
        assert choice2 == choice and np.allclose(ms2, ms, rtol=1e-3)
    finally:
        bd.psdp_destroy(h)
    with open(cache) as fh:
        assert len(fh.read().strip().splitlines()) == 1


def test_autotune_over_engines_and_tiles(bd, tmp_path):
    """psdp_autotune_ex over all six step configurations (FP64 automatic, the two
    mixed panel widths, FP64-FMA, Ozaki, Ozaki Schur with FP64-FMA Cholesky):
    the applied choice is the fastest timed one and the tuned context solves to
    the oracle's verdict; the cache answers the same shape and mask."""
    w = synth.WORKLOADS["mid"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    cache = os.path.join(tmp_path, "tune_ex.txt")
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        choice, ms = bd.psdp_autotune_ex(h, 0b111111, cache)
        assert 0 <= choice < 6 and np.all(ms > 0) and ms[choice] == ms.min()
        status, iters, info = bd.psdp_solve(h)
        assert bd.STATUS[status] == "OK" and bd.psdp_certify(h)[0] == 1
    finally:
        bd.psdp_destroy(h)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        choice2, ms2 = bd.psdp_autotune_ex(h, 0b111111, cache)
        assert choice2 == choice and np.allclose(ms2, ms, rtol=1e-3)
    finally:
        bd.psdp_destroy(h)
    # each FP64 engine configuration on its own solves to the same verdict
    for cand in (3, 4, 5):
        h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
        try:
            assert bd.psdp_autotune_ex(h, 1 << cand)[0] == cand
            status, iters, info = bd.psdp_solve(h)
            assert bd.STATUS[status] == "OK" and bd.psdp_certify(h)[0] == 1, cand
        finally:
            bd.psdp_destroy(h)
