"""Largest certifiable uncertainty set by bisection (Sec. V, Examples 1 and 2).

The uncertain system is A(beta) = sum_gamma A_gamma beta^gamma, homogeneous
of degree d_a, on an uncertainty set S_s that is the image of the unit simplex
under a linear map beta = M(s) alpha depending on a scale s.  Certifying
A'(alpha) = A(M(s) alpha) on the simplex with the library (setup, solve,
certify) certifies A on S_s.  The certified scales form an interval (a larger
set is harder), so the boundary is located by bisection, or by multisection
with several trial scales solved together in one batched launch per Newton
iteration.

Every solve runs in the library; this module only forms the coefficients of
A(M alpha) on the host and drives the search.
"""

from __future__ import annotations

from math import factorial

import numpy as np

from . import binding as bd


def monomials(l: int, d: int) -> list[tuple[int, ...]]:
    """W_d in the paper's lexicographic order, (d, 0, ..., 0) first."""
    if l == 1:
        return [(d,)]
    out = []
    for first in range(d, -1, -1):
        for rest in monomials(l - 1, d - first):
            out.append((first,) + rest)
    return out


def _power_of_linear_form(row: np.ndarray, e: int) -> dict:
    """(sum_j row_j alpha_j)^e by the multinomial theorem: exponent -> coefficient."""
    l = row.shape[0]
    out = {}
    for mu in monomials(l, e):
        c = float(factorial(e))
        for j in range(l):
            c /= factorial(mu[j])
            c *= row[j] ** mu[j]
        if c != 0.0:
            out[mu] = c
    return out


def _poly_mul(p: dict, q: dict) -> dict:
    out = {}
    for a, u in p.items():
        for b, v in q.items():
            k = tuple(x + y for x, y in zip(a, b))
            out[k] = out.get(k, 0.0) + u * v
    return out


def substitute(terms: dict, M: np.ndarray) -> np.ndarray:
    """Coefficients of A(M alpha) on W_d (lexicographic), shape [card W_d][n][n].

    terms maps exponent tuples (all of degree d) to n x n coefficients."""
    M = np.asarray(M, dtype=np.float64)
    l = M.shape[0]
    degs = {sum(e) for e in terms}
    if len(degs) != 1:
        raise ValueError("A must be homogeneous")
    d = degs.pop()
    n = next(iter(terms.values())).shape[0]
    index = {e: i for i, e in enumerate(monomials(l, d))}
    out = np.zeros((len(index), n, n))
    for e, coef in terms.items():
        poly = {tuple([0] * l): 1.0}
        for i in range(l):
            if e[i]:
                poly = _poly_mul(poly, _power_of_linear_form(M[i], e[i]))
        for k, v in poly.items():
            out[index[k]] += v * np.asarray(coef, dtype=np.float64)
    return out


def simplex_scale_map(L: float, l: int) -> np.ndarray:
    """The set S_L = {beta: sum_i beta_i = (l - 1) L + 1, L <= beta_i <= 1} of
    Example 2 (l = 3: sum = 2L + 1) as the image of the simplex:
    beta_i = (1 - L) alpha_i + L sum_j alpha_j (homogeneous of degree 1)."""
    return (1.0 - L) * np.eye(l) + L * np.ones((l, l))


def certify_scales(terms: dict, scales, map_fn, d_p: int, d1: int, precision: int = 0, eps: float = 1e-8,
                   device: int = 0) -> list[int]:
    """Verdicts (1 certified, 0 not) for each scale, all solved in one batch."""
    l = len(next(iter(terms)))
    d_a = sum(next(iter(terms)))
    hs = []
    try:
        for s in scales:
            A = substitute(terms, map_fn(s, l))
            n = A.shape[-1]
            opts = bd.psdp_default_opts(d_a=d_a, precision=precision, eps=eps, device=device)
            hs.append(bd.psdp_setup(n, l, d_p, d1, A, opts))
        bd.psdp_solve_batch(hs)
        return [int(bd.psdp_certify(h)[0]) for h in hs]
    finally:
        for h in hs:
            bd.psdp_destroy(h)


def bisect(terms: dict, lo: float, hi: float, d_p: int, d1: int, iters: int = 12, map_fn=None, **kw):
    """Smallest certified scale in [lo, hi] to within (hi - lo) / 2^iters, for
    sets that grow as the scale decreases (certified at hi, not at lo).
    Returns (bound, trace of (scale, verdict))."""
    map_fn = map_fn or simplex_scale_map
    trace = []
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        v = certify_scales(terms, [mid], map_fn, d_p, d1, **kw)[0]
        trace.append((mid, v))
        if v:
            hi = mid
        else:
            lo = mid
    return hi, trace


def multisection(terms: dict, lo: float, hi: float, d_p: int, d1: int, points: int = 7, rounds: int = 4,
                 map_fn=None, **kw):
    """As bisect, with `points` interior scales per round solved together (one
    batched launch per Newton iteration); the interval shrinks by points + 1
    per round.  Returns (bound, trace)."""
    map_fn = map_fn or simplex_scale_map
    trace = []
    for _ in range(rounds):
        grid = [lo + (hi - lo) * (k + 1) / (points + 1) for k in range(points)]
        ver = certify_scales(terms, grid, map_fn, d_p, d1, **kw)
        trace.extend(zip(grid, ver))
        new_lo, new_hi = lo, hi
        for s, v in zip(grid, ver):       # ascending: the first certified point closes the interval
            if v:
                new_hi = s
                break
            new_lo = s
        lo, hi = new_lo, new_hi
    return hi, trace
