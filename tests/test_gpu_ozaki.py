"""FP64 products by the Ozaki scheme on the BF16 tensor cores (Ozaki, Ogita,
Oishi & Rump 2012) against an accurate reference.

The reference is the compensated dot product Dot2 of Ogita, Rump & Oishi
("Accurate sum and dot product", SIAM J. Sci. Comput. 2005): error-free
products by Veltkamp splitting and error-free sums, accurate to about one
rounding of the result for these well-conditioned data.  The bound the Ozaki
product must meet follows from its construction: each entry is represented to
2^-57 of its row's power-of-two scale 2^e (max |row| < 2^e <= 2 max |row|), so
a product to 2^-56 of 2^(e_i + f_j); the levels t > 9 left out carry less than
7.1 2^-58 of it per k; the slice products are exact (every level sum an integer
below 2^24 over a depth window of 384); and the combination rounds once, plus
one rounding against the reference, so
|D_oz - D| <= K 2.8 2^(e_i + f_j - 56) + 2^-52 |D|.
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


def _split(x):
    c = 134217729.0 * x                    # 2^27 + 1
    hi = c - (c - x)
    return hi, x - hi


def dot2(A, B):
    """sum_k A[:, k] B[:, k]^T with error-free transformations (Dot2)."""
    M, N = A.shape[0], B.shape[0]
    s = np.zeros((M, N))
    c = np.zeros((M, N))
    for k in range(A.shape[1]):
        a = A[:, k][:, None]
        b = B[:, k][None, :]
        p = a * b
        ah, al = _split(a)
        bh, bl = _split(b)
        e = al * bl - (((p - ah * bh) - al * bh) - ah * bl)
        t = s + p
        z = t - s
        c += ((s - (t - z)) + (p - z)) + e
        s = t
    return s + c


def _scale(A):
    """2^e per row: the power of two just above the row's largest magnitude."""
    m = np.abs(A).max(axis=1)
    return np.ldexp(1.0, np.frexp(m)[1]) * (m > 0)


def _bound(A, B, D):
    """Deeper than 384 the product is formed in windows of 384, each within the
    bound above, and the windows are summed in FP64 (one rounding each)."""
    K = A.shape[1]
    windows = -(-K // 384)
    extra = (windows - 1) * 2.0 ** -52 * (np.abs(A) @ np.abs(B).T) if windows > 1 else 0.0
    return K * 2.8 * 2.0 ** -56 * _scale(A)[:, None] * _scale(B)[None, :] + 2.0 ** -52 * np.abs(D) + extra


@pytest.mark.parametrize("M,N,K", [(300, 200, 256), (129, 65, 70), (128, 64, 32), (40, 300, 1), (257, 130, 200),
                                   (100, 90, 600), (200, 140, 384), (130, 70, 800)])
def test_ozaki_product_is_fp64_accurate(bd, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(N, K))
    got = bd.psdp_ozaki_gemm_check(A, B)
    ref = dot2(A, B)
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= _bound(A, B, ref))
    # at least as accurate as the plain FP64 product, within its own bound
    assert np.all(np.abs(got - A @ B.T) <= K * 2.0 ** -52 * (np.abs(A) @ np.abs(B).T) + _bound(A, B, ref))


def test_ozaki_wide_dynamic_range(bd):
    """Rows of very different scales (1e-8 .. 1e8) and entries spread over six
    decades within a row: the per-row scaling keeps each row's accuracy."""
    rng = np.random.default_rng(5)
    M, N, K = 192, 160, 256
    A = rng.normal(size=(M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, K)) * 10.0 ** rng.uniform(-8, 8, size=(M, 1))
    B = rng.normal(size=(N, K)) * 10.0 ** rng.uniform(-3, 3, size=(N, K)) * 10.0 ** rng.uniform(-8, 8, size=(N, 1))
    got = bd.psdp_ozaki_gemm_check(A, B)
    ref = dot2(A, B)
    assert np.all(np.abs(got - ref) <= _bound(A, B, ref))


def test_ozaki_level_sums_near_the_exactness_limit(bd):
    """Every entry x = -64 (128^7 + ... + 1) 2^-56 (row scale 2^0), whose eight
    balanced digits are all -64: every slice product is 4096 with one sign, so
    the level sums reach (t - 1) 4096 K, 12.6 M < 2^24 at the full depth 384.
    A tensor-core accumulation that rounded near 2^24 would miss the bound by
    far (a level-2 unit is 2^-14 of the scale)."""
    X = -64 * sum(128 ** j for j in range(8))
    x = X / 2.0 ** 56
    assert x * 2.0 ** 56 == X
    for K in (384, 383, 768):
        A = np.full((130, K), x)
        B = np.full((70, K), x)
        got = bd.psdp_ozaki_gemm_check(A, B)
        ref = dot2(A, B)
        assert np.all(np.abs(got - ref) <= _bound(A, B, ref))


def test_ozaki_integer_products_are_exact(bd):
    """Small integers: every step is exact, so the result is the exact product."""
    rng = np.random.default_rng(6)
    A = rng.integers(-1000, 1001, size=(150, 256)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(90, 256)).astype(np.float64)
    got = bd.psdp_ozaki_gemm_check(A, B)
    assert np.array_equal(got, A @ B.T)


def test_ozaki_lower_update(bd):
    """C <- C - A B^T on the elements with i >= j only (the Cholesky trailing update form)."""
    rng = np.random.default_rng(7)
    M, K = 300, 128
    P = rng.normal(size=(M, K))
    C0 = rng.normal(size=(M, M))
    got = bd.psdp_ozaki_gemm_check(P, P, C0, alpha=-1.0, beta=1.0, lower=True)
    ref = C0 - dot2(P, P)
    low = np.tril(np.ones((M, M), dtype=bool))
    assert np.array_equal(got[~low], C0[~low])
    err = np.abs(got - ref)[low]
    assert np.all(err <= (_bound(P, P, ref) + 2.0 ** -52 * np.abs(C0))[low])


def test_fp64_peaks(bd):
    dfma, dmma = bd.psdp_fp64_peaks(0)
    assert 0.2 < dfma < 5.0 and 0.2 < dmma < 5.0
