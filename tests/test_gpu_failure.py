"""Failure detection without a GPU fault: a bounded device wait that runs out
reports ETIMEOUT to the host and leaves the context usable."""

import pytest

from paper_1411_3769_gb300 import synth

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


def test_unset_ready_flag_times_out_and_device_stays_usable(bd):
    status, ms = bd.psdp_trsv_timeout_check()
    assert status == "ETIMEOUT"
    assert 1900.0 <= ms <= 20000.0            # the 2 s limit, not a hang
    # the same process keeps solving afterwards
    w = synth.WORKLOADS["tiny"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    with bd.Solver(A, w["d_p"], w["d1"]) as s:
        st, it, info = s.solve()
        assert st == "OK" and s.certify()[0] == 1
