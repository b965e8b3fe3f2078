"""Learned warm start for a family of Polya SDPs (driver; every computation
runs in the library: solves, training, inference, start repair).

Family: fixed (n, l, d_p, d1), systems drawn by ``synth.system`` with the
uncertainty scale s uniform in a range.  Features are the flattened
A_1..A_l; targets are the optimal dual y* (K values) and log(tr(X*_g) / n) per
block (L + M values).  A prediction becomes a start through ``psdp_set_start``
(y0, X_g = exp(pred_g) I, Z lifted to lambda_min >= theta / x_g); the plain
cold start is the fallback whenever the warm-started solve does not end in the
same kind of outcome, and the cold solve is the judge of every verdict.
"""

from __future__ import annotations

import time

import numpy as np

from . import binding as bd
from . import synth

THETA = 0.1


def draw(count: int, n: int, l: int, s_range, base_seed: int):
    rng = np.random.default_rng(base_seed)
    out = []
    for i in range(count):
        s = float(rng.uniform(*s_range))
        out.append((synth.system(n, l, s, base_seed + 1 + i), s))
    return out


def solve_family(systems, d_p: int, d1: int, precision: int = 1, eps: float = 1e-7):
    """Solve every system (one batched launch per iteration); returns features,
    targets, statuses, iteration counts and verdicts."""
    handles = [bd.psdp_setup(A.shape[-1], A.shape[0], d_p, d1, A, bd.psdp_default_opts(precision=precision, eps=eps))
               for A, _ in systems]
    try:
        status, iters = bd.psdp_solve_batch(handles)
        feats, targs, verdicts = [], [], []
        for h, (A, _) in zip(handles, systems):
            X, Z, y = bd.psdp_get_iterate(h)
            n = A.shape[-1]
            xs = np.log(np.maximum(np.einsum("gii->g", X) / n, 1e-30))
            feats.append(A.reshape(-1))
            targs.append(np.concatenate([y, xs]))
            verdicts.append(bd.psdp_certify(h)[0])
    finally:
        for h in handles:
            bd.psdp_destroy(h)
    return (np.array(feats, np.float32), np.array(targs, np.float32), status, np.array(iters),
            np.array(verdicts))


def train(feats, targs, width: int = 1024, epochs: int = 200, batch: int = 64, lr: float = 1e-3, seed: int = 0):
    n_in, n_out = feats.shape[1], targs.shape[1]
    m = bd.psdp_mlp_create(n_in, width, n_out, max(batch, 8), seed)
    loss = bd.psdp_mlp_train(m, feats, targs, epochs, batch, lr, seed)
    return m, loss


def solve_warm(m, A, d_p: int, d1: int, K: int, nblk: int, precision: int = 1, eps: float = 1e-7):
    """Warm-started solve; falls back to the cold start if the warm run fails."""
    pred = bd.psdp_mlp_predict(m, A.reshape(1, -1).astype(np.float32), K + nblk)[0].astype(np.float64)
    with bd.Solver(A, d_p, d1, precision=precision, eps=eps) as s:
        bd.psdp_set_start(s.h, pred[:K], np.exp(np.clip(pred[K:], -30, 30)), THETA)
        status, iters, info = s.solve()
        verdict = s.certify()[0]
        fallback = False
        if status not in ("OK", "EUNBOUNDED"):
            fallback = True
    if fallback:
        with bd.Solver(A, d_p, d1, precision=precision, eps=eps) as s:
            status, it2, info = s.solve()
            verdict = s.certify()[0]
            iters += it2
    return status, iters, verdict, fallback


def evaluate(m, systems, d_p: int, d1: int, precision: int = 1, eps: float = 1e-7):
    """Cold vs warm solves of held-out systems: iterations, verdicts, wall time."""
    cold_it, warm_it, agree, fallbacks, t_cold, t_warm = [], [], [], 0, 0.0, 0.0
    for A, _ in systems:
        t0 = time.perf_counter()
        with bd.Solver(A, d_p, d1, precision=precision, eps=eps) as s:
            st_c, it_c, _ = s.solve()
            v_c = s.certify()[0]
            K, nblk = s.sizes["K"], s.sizes["nblk"]
        t1 = time.perf_counter()
        st_w, it_w, v_w, fb = solve_warm(m, A, d_p, d1, K, nblk, precision, eps)
        t2 = time.perf_counter()
        t_cold += t1 - t0
        t_warm += t2 - t1
        cold_it.append(it_c)
        warm_it.append(it_w)
        agree.append(v_c == v_w)
        fallbacks += int(fb)
    return dict(cold_iters=float(np.mean(cold_it)), warm_iters=float(np.mean(warm_it)),
                iterations_saved=float(np.mean(cold_it) - np.mean(warm_it)), verdicts_agree=bool(all(agree)),
                fallbacks=fallbacks, cold_s=t_cold, warm_s=t_warm, count=len(systems))
