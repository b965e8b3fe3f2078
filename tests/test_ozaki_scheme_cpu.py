"""The arithmetic the Ozaki-scheme kernels rely on (Ozaki, Ogita, Oishi & Rump
2012), restated on the host in exact integer arithmetic, independent of the
kernels:

* the split: X = round(x 2^(56-e)) (max |row| < 2^e) written in eight
  balanced base-128 digits, s_1 in [-128, 128] and s_2..s_8 in [-64, 63], each
  an integer of at most 8 significant bits (exact in BF16);
* the level sums T_t = sum_{p+q=t} sum_k s_p(a_k) s_q(b_k), t = 2..9, stay
  integers below 2^24 in magnitude over a depth window of 384, so an FP32
  accumulation of them is exact;
* the combination 2^(e+f-63) (Va 2^28 + Vb), Va = T_2 128^3 + ... + T_5,
  Vb = T_6 128^3 + ... + T_9, is the product of the rounded rows without the
  levels t > 9, whose pairs have digits of at most 64, so per k they carry at
  most 2^12 (7 2^-70 + 6 2^-77 + ...) < 7.1 2^-58 of the scale 2^(e+f);
* so the error of an element is at most K 2.8 2^(e+f-56) + 2^-53 |D|: 2^-56 of
  the scale per k from the split, 7.1 2^-58 from the levels left out, one
  rounding of the combination.
"""

import math
import random

import numpy as np
import pytest

WINDOW = 384


def split_row(x):
    """Digits of every entry of one row and the row exponent e."""
    m = max(abs(v) for v in x)
    e = math.frexp(m)[1] if m > 0 else 0                # m < 2^e
    digits = []
    for v in x:
        X = round(math.ldexp(v, 56 - e))                # exact: a double times a power of two, then RNE
        d = [0] * 8
        for p in range(7, 0, -1):
            r = ((X + 64) & 127) - 64
            d[p] = r
            X = (X - r) >> 7
        d[0] = X
        digits.append(d)
    return digits, e


def levels(da, db):
    """Level sums T_2..T_9 of two rows of digits (exact Python integers)."""
    T = [0] * 8
    for sa, sb in zip(da, db):
        for p in range(8):
            for q in range(8 - p):
                T[p + q] += sa[p] * sb[q]
    return T


def check_bf16_exact(d):
    a = abs(d)
    return a == 0 or (a >> max(0, a.bit_length() - 8)) << max(0, a.bit_length() - 8) == a


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_digits_reconstruct_and_fit_bf16(seed):
    rng = random.Random(seed)
    x = [rng.uniform(-1, 1) * 2.0 ** rng.randint(-30, 30) for _ in range(200)]
    digits, e = split_row(x)
    for v, d in zip(x, digits):
        X = sum(s * 128 ** (7 - p) for p, s in enumerate(d))
        assert X == round(math.ldexp(v, 56 - e))
        assert -128 <= d[0] <= 128 and all(-64 <= s <= 63 for s in d[1:])
        assert all(check_bf16_exact(s) for s in d)
        # the representation error is at most half a unit of 2^(e-56)
        assert abs(math.ldexp(X, e - 56) - v) <= math.ldexp(1.0, e - 57)


def test_level_sums_stay_below_two_to_the_24_at_the_window():
    # the worst case: every digit -64 (products 4096, one sign), and the first digit 128
    X = -64 * sum(128 ** j for j in range(8))
    x = X / 2.0 ** 56
    digits, e = split_row([x] * WINDOW)
    assert all(s == -64 for s in digits[0])
    T = levels(digits, digits)
    assert max(abs(t) for t in T) == 8 * 4096 * WINDOW        # level 9: eight pairs
    assert max(abs(t) for t in T) < 2 ** 24
    # the bound the kernel states, 10 * 2^12 per k, covers a first digit of 128 too
    assert 10 * 2 ** 12 * WINDOW < 2 ** 24 <= 10 * 2 ** 12 * (WINDOW + 32)
    big = [128] + [63] * 7
    T = levels([big] * WINDOW, [big] * WINDOW)
    assert max(abs(t) for t in T) < 2 ** 24


@pytest.mark.parametrize("seed", [3, 4])
def test_combination_is_the_truncated_exact_product(seed):
    rng = np.random.default_rng(seed)
    K = 97
    a = list(rng.normal(size=K) * 10.0 ** rng.uniform(-3, 3, size=K))
    b = list(rng.normal(size=K) * 10.0 ** rng.uniform(-3, 3, size=K))
    da, e = split_row(a)
    db, f = split_row(b)
    T = levels(da, db)
    Va = ((T[0] * 128 + T[1]) * 128 + T[2]) * 128 + T[3]
    Vb = ((T[4] * 128 + T[5]) * 128 + T[6]) * 128 + T[7]
    assert abs(Va) < 2 ** 53 and abs(Vb) < 2 ** 53             # exact in FP64
    # the exact product of the rounded rows, in units of 2^(e+f-112)
    Xa = [sum(s * 128 ** (7 - p) for p, s in enumerate(d)) for d in da]
    Xb = [sum(s * 128 ** (7 - p) for p, s in enumerate(d)) for d in db]
    exact = sum(u * v for u, v in zip(Xa, Xb))
    kept = (Va * 2 ** 28 + Vb) * 2 ** 49                       # levels t <= 9, same units
    dropped = exact - kept
    # the dropped levels t >= 10: less than 7.1 2^-58 of the scale per k, i.e.
    # K 7.1 2^54 in these units (2^(e+f-112))
    assert abs(dropped) < K * 7.1 * 2 ** 54
    # one rounding of the combination gives the kernel's value; it is within the
    # stated bound of the true product
    D = math.ldexp(float(Va * 2 ** 28 + Vb), e + f - 63)
    true = math.fsum(u * v for u, v in zip(a, b))
    bound = K * 2.8 * math.ldexp(1.0, e + f - 56) + 2.0 ** -52 * abs(true)
    assert abs(D - true) <= bound


def test_truncation_bound_is_reached_by_the_worst_digits():
    """All digits -64 in both operands: every left-out level has all its pairs
    at 4096 with one sign, so the truncation is the stated 2^12 sum per k."""
    X = -64 * sum(128 ** j for j in range(8))
    da = [[-64] * 8]
    T_all = [0] * 15
    for p in range(8):
        for q in range(8):
            T_all[p + q] += 4096
    dropped = sum(T_all[t - 2] * 2 ** (7 * (16 - t)) for t in range(10, 17))
    per_k = 2 ** 12 * sum((17 - t) * 2 ** (7 * (16 - t)) for t in range(10, 17))
    assert dropped == per_k < 7.1 * 2 ** 54
    assert X * X == sum(T_all[t - 2] * 2 ** (7 * (16 - t)) for t in range(2, 17))
    assert levels(da, da)[7] == 8 * 4096
