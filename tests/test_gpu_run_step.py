"""The step-timing entry point (python -m paper_1411_3769_gb300.run_step) on the
tiny workload, in both precisions and with each FP64 engine."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def run_step():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_3769_gb300 import run_step
    return run_step


@pytest.mark.parametrize("precision,engine", [("fp64", "auto"), ("fp64", "fma"), ("fp64", "ozaki"), ("mixed", "auto")])
def test_run_step_reports_a_step(run_step, precision, engine):
    out = run_step.main(["--workload", "tiny", "--precision", precision, "--engine", engine, "--steps", "2",
                         "--warmup", "1"])
    assert out["workload"] == "tiny" and len(out["ms"]) == 2 and out["ms_per_step"] > 0
    assert out["kernels_per_step"] > 0
    want = {"fma": "dfma", "ozaki": "ozaki"}.get(engine)
    if want:
        assert out["engines"] == {"schur": want, "cholesky": want}
