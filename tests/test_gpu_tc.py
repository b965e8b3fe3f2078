"""The tcgen05 tensor-core GEMM against an FP64 product of the same operands.

TF32 (split 1): the operands are first rounded to TF32 on the host (10-bit
mantissa; the tensor core drops the low 13 bits, so host rounding to nearest
may differ by one TF32 ulp), so the bound is a few TF32 ulps of sum |a||b|.
3xTF32 (split 3): the hi*hi + hi*lo + lo*hi product keeps about 2^-21 of each
term, bound 1e-5 * sum |a||b| (FP32 accumulation over K adds K*2^-24).
BF16: operands exact in BF16, FP32 accumulation: bound K * 2^-23 * sum |a||b|.
"""

import numpy as np
import pytest

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


def _tf32(x):
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def _bf16_bits(x):
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def _bf16_val(b):
    return (b.astype(np.uint32) << 16).view(np.float32)


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 200, 100), (64, 500, 7), (257, 129, 333)])
def test_tf32(bd, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    D = bd.psdp_tc_gemm_check(A, B, split=1)
    ref = _tf32(A).astype(np.float64) @ _tf32(B).astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    assert np.all(np.abs(D - ref) <= 4 * 2.0 ** -10 * scale + 1e-6)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 100), (129, 257, 500)])
def test_3xtf32(bd, M, N, K):
    rng = np.random.default_rng(7 + M)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    D = bd.psdp_tc_gemm_check(A, B, split=3)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    err = np.abs(D - ref) / scale
    assert err.max() <= 1e-5
    # and clearly better than plain TF32 (the split terms are really used)
    D1 = bd.psdp_tc_gemm_check(A, B, split=1)
    assert err.max() < 0.1 * (np.abs(D1 - ref) / scale).max()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 512), (200, 100, 70)])
def test_bf16(bd, M, N, K):
    rng = np.random.default_rng(11 + K)
    A = _bf16_bits(rng.normal(size=(M, K)))
    B = _bf16_bits(rng.normal(size=(N, K)))
    D = bd.psdp_tc_gemm_check(A, B)
    Af, Bf = _bf16_val(A).astype(np.float64), _bf16_val(B).astype(np.float64)
    ref = Af @ Bf.T
    scale = np.abs(Af) @ np.abs(Bf).T
    assert np.all(np.abs(D - ref) <= K * 2.0 ** -23 * scale + 1e-6)


@pytest.mark.parametrize("M,N,K,split,tri,ctas", [
    (1000, 1000, 128, 3, 1, 152),   # trailing update shape, one tile per CTA at most
    (1000, 1000, 128, 3, 1, 5),     # five CTAs walk 36 tiles: accumulator double buffer and stage ring wrap
    (700, 128, 128, 3, 1, 3),       # next-panel strip (one tile column)
    (300, 500, 100, 1, 0, 4),       # full update, ragged K and tiles, plain TF32
    (257, 257, 64, 3, 1, 2),
])
def test_persistent_update(bd, M, N, K, split, tri, ctas):
    """C - A B^T on the selected tiles; the tiles outside are untouched."""
    rng = np.random.default_rng(M + 3 * K + ctas)
    A = rng.normal(size=(M, K)).astype(np.float32)
    B = rng.normal(size=(N, K)).astype(np.float32)
    C0 = rng.normal(size=(M, N)).astype(np.float32)
    out = bd.psdp_tc_gemm_persist_check(A, B, C0, split=split, tri=tri, ctas=ctas)
    mt = (np.arange(M) // 128)[:, None]
    nt = (np.arange(N) // 128)[None, :]
    sel = (mt >= nt) if tri else np.ones((M, N), bool)
    if split == 3:
        prod = A.astype(np.float64) @ B.astype(np.float64).T
        tol = 1e-5
    else:
        prod = _tf32(A).astype(np.float64) @ _tf32(B).astype(np.float64).T
        tol = 4 * 2.0 ** -10
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T + np.abs(C0)
    ref = C0.astype(np.float64) - prod
    assert np.all(np.abs(out - ref)[sel] <= tol * scale[sel] + 1e-5)
    assert np.array_equal(out[~sel], C0[~sel])
