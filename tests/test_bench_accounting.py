"""The algorithmic work the bench's roofline divides by.  However the per-kernel
FP64 flop counts of the Cholesky group the trailing updates (inner, block,
next-panel, bulk), they must add up exactly to the right-looking
factorization's: each 32-column panel of width w updates the lower triangle of
the rest x rest trailing matrix, w rest (rest + 1) flops, ~K^3/3 in all
(Sec. IV-C: the root's Cholesky of Omega); the panel solves add 2 rest w^2."""

import pytest

import bench


def _right_looking(K, w=32):
    upd = trsm = 0.0
    for j0 in range(0, K, w):
        rest = K - j0 - min(w, K - j0)
        upd += min(w, K - j0) * rest * (rest + 1.0)
        trsm += 2.0 * rest * min(w, K - j0) ** 2
    return upd, trsm


@pytest.mark.parametrize("K", [630, 2100, 4920, 8192, 10980, 30300])
def test_ozaki_cholesky_flops_add_up(K):
    cf = bench.chol_flops_ozaki(K)
    assert set(cf) == {"trsm", "inner", "block", "next", "bulk"}
    upd, trsm = _right_looking(K)
    assert abs(sum(cf.values()) - cf["trsm"] - upd) <= 1e-9 * upd
    assert abs(cf["trsm"] - trsm) <= 1e-9 * trsm
    assert abs(upd - K ** 3 / 3) <= 0.1 * K ** 3 / 3
    if K < 8192:
        assert cf["block"] == 0.0 and bench.oz_outer(K) == 256
    else:
        assert cf["block"] > 0.0 and bench.oz_outer(K) == bench.OZ_DEPTH == 384


@pytest.mark.parametrize("K", [2100, 30300])
def test_fma_cholesky_flops_add_up(K):
    cf = bench.chol_flops(K, 32)
    upd, trsm = _right_looking(K)
    assert abs(sum(cf.values()) - cf["trsm"] - upd) <= 1e-9 * upd


def test_ozaki_traffic_per_element_is_the_c_update_and_slices():
    # C read and written once (16 B an element) plus the slices: between 16 and 20 B
    assert 16.0 < bench.OZ_DRAM_BYTES_PER_ELEMENT < 20.0
