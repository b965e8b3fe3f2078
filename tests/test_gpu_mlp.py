"""BF16 tensor-core MLP against the FP64 oracle MLP, and the learned warm start.

Gradient tolerances.  The GPU multiplies BF16 operands (8 significant bits,
unit roundoff u = 2^-9) with FP32 accumulation (2^-24) and rounds each hidden
activation and each back-propagated gradient to BF16 before the next product.
(1) Against a reference that rounds at exactly those points (FP64 otherwise)
only the FP32 accumulation order differs: bound 1e-3 per tensor in the
Frobenius norm.  (2) Against the plain FP64 oracle fed the same BF16-rounded
weights and inputs the roundings themselves show.  `_error_bound` carries a
first-order bound on that difference through the network element by element:
each rounding contributes u (or 2^-24) times the magnitude it rounds, a
product passes its operands' bounds on through |W|, a ReLU is 1-Lipschitz, and
where |Z| is within its own bound the mask of the backward pass may flip, which
contributes the whole |g||W| there.  The test allows twice that bound, for the
second-order terms (u^2 relative) the first-order bound leaves out.
The warm start must keep every verdict of the cold solve and, on average, take fewer interior-point iterations.
"""

import numpy as np
import pytest

from oracle import mlp as omlp

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


def _bf16(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _faithful(params, X, T):
    """Forward/backward in FP64 with BF16 rounding where the GPU rounds."""
    H = [_bf16(X)]
    Z = []
    for i, (W, b) in enumerate(params):
        z = H[-1] @ _bf16(W).T + b
        Z.append(z)
        if i < len(params) - 1:
            H.append(_bf16(np.maximum(z, 0.0)))
    g = 2.0 * (Z[-1] - T) / T.size
    grads = [None] * len(params)
    for i in range(len(params) - 1, -1, -1):
        gb = g.sum(axis=0)
        gq = _bf16(g)
        grads[i] = [gq.T @ H[i], gb]
        if i > 0:
            g = (gq @ _bf16(params[i][0])) * (Z[i - 1] > 0.0)
    return grads


U_BF16 = 2.0 ** -9
U_FP32 = 2.0 ** -24


def _error_bound(params, X, T):
    """First-order elementwise bound on |GPU gradient - FP64 gradient| for the
    rounding points described in the module docstring (weights already BF16)."""
    H, eH, Z, eZ = [_bf16(X)], [np.zeros(X.shape)], [], []
    nl = len(params)
    for i, (W, b) in enumerate(params):
        aW = np.abs(W)
        k = W.shape[1]
        z = H[-1] @ W.T + b
        Z.append(z)
        eZ.append(eH[-1] @ aW.T + (k + 1) * U_FP32 * (np.abs(H[-1]) @ aW.T + np.abs(b)))
        if i < nl - 1:
            h = np.maximum(z, 0.0)
            H.append(h)
            eH.append(eZ[-1] + U_BF16 * h)
    g = 2.0 * (Z[-1] - T) / T.size
    eg = 2.0 * eZ[-1] / T.size + U_FP32 * np.abs(g)
    B = X.shape[0]
    out = [None] * nl
    for i in range(nl - 1, -1, -1):
        egq = eg + U_BF16 * np.abs(g)
        eW = egq.T @ np.abs(H[i]) + np.abs(g).T @ eH[i] + (B + 1) * U_FP32 * (np.abs(g).T @ np.abs(H[i]))
        eb = eg.sum(axis=0) + B * U_FP32 * np.abs(g).sum(axis=0)
        out[i] = [eW, eb]
        if i > 0:
            W = params[i][0]
            aW = np.abs(W)
            mask = Z[i - 1] > 0.0
            flip = np.abs(Z[i - 1]) <= eZ[i - 1]
            eg = (egq @ aW) * mask + flip * (np.abs(g) @ aW) + (W.shape[0] + 1) * U_FP32 * (np.abs(g) @ aW)
            g = (g @ W) * mask
    loss_bound = np.mean(2.0 * np.abs(Z[-1] - T) * eZ[-1]) + T.size * U_FP32 * np.mean((Z[-1] - T) ** 2)
    return out, loss_bound


def _unflat(flat, sizes):
    out, off = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = flat[off:off + a * b].reshape(b, a)
        off += a * b
        bb = flat[off:off + b]
        off += b
        out.append([W, bb])
    return out


@pytest.mark.parametrize("sizes,B", [((16, 32, 32, 10), 8), ((64, 128, 128, 37), 40)])
def test_gradients_match_oracle(bd, sizes, B):
    n_in, width, _, n_out = sizes
    h = bd.psdp_mlp_create(n_in, width, n_out, max(B, 8), seed=3)
    try:
        rng = np.random.default_rng(4)
        X = rng.normal(size=(B, n_in)).astype(np.float32)
        T = rng.normal(size=(B, n_out)).astype(np.float32)
        flat = bd.psdp_mlp_params(h).astype(np.float64)
        loss, g = bd.psdp_mlp_grads(h, X, T)
        params = _unflat(flat, sizes)
        for p in params:
            p[0] = _bf16(p[0])
        Y, cache = omlp.forward(params, _bf16(X))
        ref = omlp.backward(params, cache, Y, T.astype(np.float64))
        bound, loss_bound = _error_bound(params, X.astype(np.float64), T.astype(np.float64))
        assert abs(loss - omlp.loss(Y, T)) <= 2.0 * loss_bound
        gp = _unflat(g.astype(np.float64), sizes)
        for (gw, gb), (rw, rb), (ew, eb) in zip(gp, ref, bound):
            assert np.all(np.abs(gw - rw) <= 2.0 * ew + 1e-12)
            assert np.all(np.abs(gb - rb) <= 2.0 * eb + 1e-12)
        fa = _faithful(_unflat(flat, sizes), X.astype(np.float64), T.astype(np.float64))
        for (gw, gb), (rw, rb) in zip(gp, fa):
            assert np.linalg.norm(gw - rw) <= 1e-3 * np.linalg.norm(rw) + 1e-7
            assert np.linalg.norm(gb - rb) <= 1e-3 * np.linalg.norm(rb) + 1e-7
    finally:
        bd.psdp_mlp_destroy(h)


def test_training_reduces_loss(bd):
    rng = np.random.default_rng(5)
    Wt = rng.normal(size=(24, 16))
    X = rng.normal(size=(512, 16)).astype(np.float32)
    T = np.tanh(X @ Wt.T).astype(np.float32)
    h = bd.psdp_mlp_create(16, 64, 24, 64, seed=1)
    try:
        l1 = bd.psdp_mlp_train(h, X, T, epochs=1, batch=64, lr=1e-3)
        l2 = bd.psdp_mlp_train(h, X, T, epochs=60, batch=64, lr=1e-3)
        assert l2 < 0.3 * l1
        Y = bd.psdp_mlp_predict(h, X[:50], 24)
        assert np.mean((Y - T[:50]) ** 2) < 0.3 * np.mean(T[:50] ** 2)
    finally:
        bd.psdp_mlp_destroy(h)


def test_warm_start_keeps_verdicts_and_saves_iterations(bd):
    from paper_1411_3769_gb300 import warmstart as ws
    n, l, d_p, d1 = 6, 2, 1, 1
    train_sys = ws.draw(96, n, l, (0.1, 0.8), base_seed=100)
    test_sys = ws.draw(12, n, l, (0.1, 0.8), base_seed=900)
    F, T, status, iters, verdicts = ws.solve_family(train_sys, d_p, d1, stop_iter=ws.K_TARGET)
    ok = np.array([s in ("OK", "EMAXITER") for s in status])
    assert ok.sum() >= 48
    m, loss = ws.train(F[ok], T[ok], width=128, epochs=300, batch=16, lr=1e-3)
    try:
        res = ws.evaluate(m, test_sys, d_p, d1)
    finally:
        bd.psdp_mlp_destroy(m)
    assert res["verdicts_agree"]
    assert res["warm_iters"] < res["cold_iters"]
