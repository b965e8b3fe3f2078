"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only draws the system
matrices A_1..A_l of an affine uncertain system A(alpha) = sum_i A_i alpha_i
on the simplex, shaped like the paper's random test systems (Sec. V,
Example 3).  Generator (numpy PCG64 ``default_rng(seed)``, draw order M then
E_1..E_l):

    M_ij ~ N(0, 1/n),  A0 = M - (max Re eig(M) + 1) I,
    E_i  ~ N(0, 1/n),  A_i = A0 + s E_i.

A0 is Hurwitz with spectral abscissa -1; the uncertainty scale s moves the
vertices A_i away from it, so small s gives robustly stable systems and large
s (typically) unstable ones.  Arrays are float64, shape (l, n, n), row-major.
"""

from __future__ import annotations

import numpy as np


def system(n: int, l: int, s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    M = rng.normal(0.0, 1.0 / np.sqrt(n), size=(n, n))
    A0 = M - (np.linalg.eigvals(M).real.max() + 1.0) * np.eye(n)
    E = rng.normal(0.0, 1.0 / np.sqrt(n), size=(l, n, n))
    return np.ascontiguousarray(A0[None, :, :] + s * E)


# Named workloads: (n, l, d_p, d1) and the uncertainty scale used for them.
WORKLOADS = {
    "tiny":    dict(n=5, l=2, d_p=1, d1=1, s=0.2),     # K = 30, 7 blocks
    "tiny_unstable": dict(n=5, l=2, d_p=1, d1=1, s=2.0),
    "mid":     dict(n=20, l=4, d_p=2, d1=3, s=0.3),    # K = 2100, 140 blocks
    "large":   dict(n=100, l=3, d_p=2, d1=4, s=0.3),   # K = 30300, 64 blocks
    "warm":    dict(n=32, l=3, d_p=2, d1=3, s=0.8),    # K = 3168, 49 blocks
}


def batch_instances(count: int, base_seed: int = 1000, n_range=(8, 48)) -> list[dict]:
    """Uneven instances (bisection points on the uncertainty scale s):
    n ~ U{8..48}, l ~ U{2,3,4}, d_p ~ U{1,2}, d1 ~ U{1..4}, s ~ U[0.05, 3.0];
    instance i draws its shape from ``default_rng(base_seed + i)`` and its
    matrices from ``system(..., seed=base_seed + i)``."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(base_seed + i)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        l = int(rng.integers(2, 5))
        d_p = int(rng.integers(1, 3))
        d1 = int(rng.integers(1, 5))
        s = float(rng.uniform(0.05, 3.0))
        out.append(dict(n=n, l=l, d_p=d_p, d1=d1, s=s, seed=base_seed + i,
                        A=system(n, l, s, base_seed + i)))
    return out
