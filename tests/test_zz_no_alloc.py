"""The allocation-free tensor-core GEMM entry point against the allocating one.

psdp_tc_gemm_noalloc serves callers that cannot allocate device memory where
they need the product (inside a global-mode graph capture, in allocator
callbacks, under a fixed device budget).  It must give the same product as
psdp_tc_gemm_check on the same inputs, on consecutive calls that reuse its
static scratch, and refuse sizes beyond that scratch.  This file is collected
last so a failure here leaves every other test already run.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_3769_gb300 import build
    build.build()
    from paper_1411_3769_gb300 import binding
    binding._lib()
    return binding, torch


def _noalloc(bd, torch, A, B, split):
    M, K = A.shape
    N = B.shape[0]
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((N, M), float("nan"), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    s = bd.psdp_tc_gemm_noalloc(M, N, K, split, dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), stream.cuda_stream)
    assert s == 0, bd.STATUS.get(s, s)
    return dC.cpu().numpy().T


@pytest.mark.parametrize("split", [3, 1])
def test_noalloc_matches_allocating_entry_point_twice(env, split):
    bd, torch = env
    rng = np.random.default_rng(split)
    for M, N, K in ((300, 200, 100), (129, 257, 70)):      # two calls in a row on the shared scratch
        A = rng.normal(size=(M, K)).astype(np.float32)
        B = rng.normal(size=(N, K)).astype(np.float32)
        got = _noalloc(bd, torch, A, B, split)
        ref = bd.psdp_tc_gemm_check(A, B, split=split)
        scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 1e-6 * scale)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    bd, torch = env
    M, N, K = 8192, 8192, 128
    kpad = (K + 63) // 64 * 64
    # the call must be refused on the host before any device access: make sure
    # the case really is beyond the scratch before handing over placeholder pointers
    assert (M + N) * kpad > 2 ** 20
    s = bd.psdp_tc_gemm_noalloc(M, N, K, 3, 1, 1, 1, 0)
    assert bd.STATUS[s] == "EINVAL"
