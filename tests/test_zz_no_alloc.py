"""The allocation-free tensor-core GEMM entry point against the allocating one.

psdp_tc_gemm_noalloc serves callers that cannot allocate device memory where
they need the product: allocator or memory-pool callbacks, where an allocation
would re-enter the allocator, and hosts that give the library a fixed device
budget.  It must give the same product as psdp_tc_gemm_check on the same
inputs, on consecutive calls that reuse its static scratch, leave the device's
free memory unchanged, and refuse sizes beyond that scratch.  This file is
collected last so a failure here leaves every other test already run.
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


def _noalloc_dev(bd, torch, dA, dB, dC, split):
    M, K = dA.shape
    N = dB.shape[0]
    stream = torch.cuda.current_stream()
    s = bd.psdp_tc_gemm_noalloc(M, N, K, split, dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), stream.cuda_stream)
    assert s == 0, bd.STATUS.get(s, s)


def _noalloc(bd, torch, A, B, split):
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((B.shape[0], A.shape[0]), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    _noalloc_dev(bd, torch, dA, dB, dC, split)
    return dC.cpu().numpy().T


@pytest.mark.parametrize("split", [3, 1])
def test_noalloc_matches_allocating_entry_point_twice(env, split):
    bd, torch = env
    rng = np.random.default_rng(split)
    # TF32 rounds each operand to 11 significant bits (2^-11 relative each);
    # 3xTF32 drops lo*lo (2^-22) and accumulates in FP32 (K * 2^-23 at worst)
    bound = 4e-3 if split == 1 else 2e-5
    for M, N, K in ((300, 200, 100), (129, 257, 70)):      # two calls in a row on the shared scratch
        A = rng.normal(size=(M, K)).astype(np.float32)
        B = rng.normal(size=(N, K)).astype(np.float32)
        got = _noalloc(bd, torch, A, B, split)
        ref = bd.psdp_tc_gemm_check(A, B, split=split)
        scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 1e-6 * scale)
        exact = A.astype(np.float64) @ B.astype(np.float64).T
        assert np.all(np.abs(got - exact) <= bound * scale)


def test_noalloc_leaves_free_device_memory_unchanged(env):
    bd, torch = env
    rng = np.random.default_rng(7)
    M, N, K = 256, 192, 96
    dA = torch.from_numpy(rng.normal(size=(M, K)).astype(np.float32)).cuda()
    dB = torch.from_numpy(rng.normal(size=(N, K)).astype(np.float32)).cuda()
    dC = torch.empty((N, M), dtype=torch.float32, device="cuda")
    _noalloc_dev(bd, torch, dA, dB, dC, 3)          # first call: the library's module is loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    held0 = torch.cuda.memory_allocated()
    for _ in range(3):
        _noalloc_dev(bd, torch, dA, dB, dC, 3)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == held0


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    bd, torch = env
    M, N, K = 8192, 8192, 128
    kpad = (K + 63) // 64 * 64
    # the call must be refused on the host before any device access; it still
    # gets real (one-element) device buffers, so a regression of that check
    # could not touch memory outside an allocation of this process
    assert (M + N) * kpad > 2 ** 20
    dA = torch.zeros(1, dtype=torch.float32, device="cuda")
    dB = torch.zeros(1, dtype=torch.float32, device="cuda")
    dC = torch.zeros(1, dtype=torch.float32, device="cuda")
    s = bd.psdp_tc_gemm_noalloc(M, N, K, 3, dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), 0)
    assert bd.STATUS[s] == "EINVAL"
