"""Learned warm start for a family of Polya SDPs (orchestration; every computation
runs in the library: solves, training, inference, start repair).

Family: fixed (n, l, d_p, d1), systems drawn by ``synth.system`` with the
uncertainty scale s uniform in a range.  Features are the flattened
A_1..A_l.  Targets describe one iterate of the plain cold-start solve: the
dual y (K values), log(tr(X_g) / n) per block (L + M values) and log mu,
mu = tr(ZX) / n_X.  With ``stop_iter`` = k the iterate is the one after k
interior-point steps from the cold start: a unique, continuous function of A
(the method is deterministic), unlike the optimal dual y*, which is not unique
on the optimal face and so is mostly not a function of A at all.  Without it
the targets come from the final iterate (the optimum).  A prediction becomes a
start through ``psdp_set_start`` (y0, X_g = exp(pred_g) I, Z lifted to
lambda_min >= theta / x_g with theta = the predicted mu); the plain cold start
is the fallback whenever the warm-started solve does not end in the same kind of
outcome, and every verdict is checked against the cold solve.
"""

from __future__ import annotations

import time

import numpy as np

from . import binding as bd
from . import synth

THETA = 0.1
# the cold-start iterate the network learns to propose: after this many steps,
# roughly a third of a cold solve on the n=32 family (4096 training systems are
# not enough to learn the optimum, which is not unique, nor a later iterate)
K_TARGET = 10


def draw(count: int, n: int, l: int, s_range, base_seed: int):
    rng = np.random.default_rng(base_seed)
    out = []
    for i in range(count):
        s = float(rng.uniform(*s_range))
        out.append((synth.system(n, l, s, base_seed + 1 + i), s))
    return out


CHUNK = 256   # instances per batched solve (bounds the device memory of the contexts)


def solve_family(systems, d_p: int, d1: int, precision: int = 1, eps: float = 1e-7, stop_iter: int | None = None):
    """Solve every system (one batched launch per iteration, CHUNK instances at
    a time), to the stopping rule or for stop_iter steps; returns features,
    targets (y, log(tr X_g / n), log mu of the last iterate), statuses,
    iteration counts and verdicts."""
    feats, targs, verdicts, status, iters = [], [], [], [], []
    for c0 in range(0, len(systems), CHUNK):
        part = systems[c0:c0 + CHUNK]
        handles = []
        try:
            for A, _ in part:
                opts = bd.psdp_default_opts(precision=precision, eps=eps)
                if stop_iter:
                    opts.max_iter = stop_iter
                handles.append(bd.psdp_setup(A.shape[-1], A.shape[0], d_p, d1, A, opts))
            st, it = bd.psdp_solve_batch(handles)
            status += list(st)
            iters += list(it)
            for h, (A, _) in zip(handles, part):
                X, Z, y = bd.psdp_get_iterate(h)
                n = A.shape[-1]
                xs = np.log(np.maximum(np.einsum("gii->g", X) / n, 1e-30))
                mu = float(np.einsum("gij,gji->", Z, X)) / (X.shape[0] * n)
                feats.append(A.reshape(-1))
                targs.append(np.concatenate([y, xs, [np.log(max(mu, 1e-30))]]))
                verdicts.append(bd.psdp_certify(h)[0])
        finally:
            for h in handles:
                bd.psdp_destroy(h)
    return (np.array(feats, np.float32), np.array(targs, np.float32), status, np.array(iters),
            np.array(verdicts))


def start_from(pred, K: int, nblk: int):
    """(y0, x-scales, theta) of a start from one predicted target row."""
    pred = np.asarray(pred, dtype=np.float64)
    y0 = pred[:K]
    xs = np.exp(np.clip(pred[K:K + nblk], -30, 30))
    theta = float(np.exp(np.clip(pred[K + nblk], np.log(1e-8), 0.0))) if pred.shape[0] > K + nblk else THETA
    return y0, xs, theta


def train(feats, targs, width: int = 1024, epochs: int = 200, batch: int = 64, lr: float = 1e-3, seed: int = 0):
    n_in, n_out = feats.shape[1], targs.shape[1]
    m = bd.psdp_mlp_create(n_in, width, n_out, max(batch, 8), seed)
    loss = bd.psdp_mlp_train(m, feats, targs, epochs, batch, lr, seed)
    return m, loss


def solve_warm(m, A, d_p: int, d1: int, K: int, nblk: int, precision: int = 1, eps: float = 1e-7):
    """Warm-started solve; falls back to the cold start if the warm run fails."""
    pred = bd.psdp_mlp_predict(m, A.reshape(1, -1).astype(np.float32), K + nblk + 1)[0]
    y0, xs, theta = start_from(pred, K, nblk)
    with bd.Solver(A, d_p, d1, precision=precision, eps=eps) as s:
        bd.psdp_set_start(s.h, y0, xs, theta)
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


def _batch_solve(part, d_p, d1, precision, eps, starts=None):
    """Solve a chunk in one batch, optionally from predicted starts; returns
    statuses, iterations and verdicts."""
    handles = []
    try:
        for k, (A, _) in enumerate(part):
            h = bd.psdp_setup(A.shape[-1], A.shape[0], d_p, d1, A, bd.psdp_default_opts(precision=precision, eps=eps))
            handles.append(h)
            if starts is not None:
                sz = bd.psdp_sizes(h)
                y0, xs, theta = start_from(starts[k], sz["K"], sz["nblk"])
                bd.psdp_set_start(h, y0, xs, theta)
        st, it = bd.psdp_solve_batch(handles)
        return list(st), list(it), [bd.psdp_certify(h)[0] for h in handles]
    finally:
        for h in handles:
            bd.psdp_destroy(h)


def cold_solves(systems, d_p: int, d1: int, precision: int = 0, eps: float = 1e-7):
    """Plain cold-start solves of the systems (batched, CHUNK at a time): wall
    seconds, iterations and verdicts; with precision 0 (FP64) the reference
    the mixed and warm-started solves are compared with."""
    t, it, verdicts, status = 0.0, [], [], []
    for c0 in range(0, len(systems), CHUNK):
        part = systems[c0:c0 + CHUNK]
        t0 = time.perf_counter()
        st, its, v = _batch_solve(part, d_p, d1, precision, eps)
        t += time.perf_counter() - t0
        it += its
        verdicts += v
        status += st
    return dict(seconds=t, iters=float(np.mean(it)), verdicts=verdicts, status=status)


def evaluate(m, systems, d_p: int, d1: int, precision: int = 1, eps: float = 1e-7, predict=None):
    """Cold vs warm solves of held-out systems (each side batched, CHUNK at a
    time): iterations, verdicts, fallbacks, wall time.  A warm solve that ends
    in neither OK nor EUNBOUNDED is repeated from the cold start (fallback), and
    its iterations count on the warm side.  predict(features, n_out) replaces
    the network's prediction when given (e.g. the training-set mean, the
    ablation without learning)."""
    cold_it, warm_it, agree, fallbacks, t_cold, t_warm, warm_v = [], [], [], 0, 0.0, 0.0, []
    for c0 in range(0, len(systems), CHUNK):
        part = systems[c0:c0 + CHUNK]
        t0 = time.perf_counter()
        st_c, it_c, v_c = _batch_solve(part, d_p, d1, precision, eps)
        t1 = time.perf_counter()
        feats = np.stack([A.reshape(-1) for A, _ in part]).astype(np.float32)
        first = bd.psdp_setup(part[0][0].shape[-1], part[0][0].shape[0], d_p, d1, part[0][0])
        sz = bd.psdp_sizes(first)
        bd.psdp_destroy(first)
        n_out = sz["K"] + sz["nblk"] + 1
        preds = (predict(feats, n_out) if predict is not None else bd.psdp_mlp_predict(m, feats, n_out)).astype(np.float64)
        st_w, it_w, v_w = _batch_solve(part, d_p, d1, precision, eps, starts=preds)
        for k, (A, _) in enumerate(part):
            if st_w[k] not in ("OK", "EUNBOUNDED"):
                fallbacks += 1
                with bd.Solver(A, d_p, d1, precision=precision, eps=eps) as s:
                    _, it2, _ = s.solve()
                    v_w[k] = s.certify()[0]
                    it_w[k] += it2
        t2 = time.perf_counter()
        t_cold += t1 - t0
        t_warm += t2 - t1
        cold_it += it_c
        warm_it += it_w
        agree += [a == b for a, b in zip(v_c, v_w)]
        warm_v += list(v_w)
    return dict(cold_iters=float(np.mean(cold_it)), warm_iters=float(np.mean(warm_it)),
                iterations_saved=float(np.mean(cold_it) - np.mean(warm_it)), verdicts_agree=bool(all(agree)),
                fallbacks=fallbacks, cold_s=t_cold, warm_s=t_warm, count=len(systems), warm_verdicts=warm_v)
