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


def test_profile_trace_orders_the_step(run_step):
    """psdp_profile_trace: one entry per timed launch of the last profiled step,
    in issue order, with end after start, the look-ahead chain on the critical
    stream and the aggregate of psdp_profile_get as the sum of the entries."""
    from paper_1411_3769_gb300 import binding as bd, synth
    w = synth.WORKLOADS["mid"]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A)
    try:
        assert bd.psdp_profile_trace(h) == []
        bd.psdp_profile_enable(h, True)
        bd.psdp_step(h)
        bd.psdp_profile_reset(h)
        bd.psdp_step(h)
        tr = bd.psdp_profile_trace(h)
        agg = bd.psdp_profile_get(h)
    finally:
        bd.psdp_destroy(h)
    assert len(tr) == sum(v[0] for v in agg.values())
    assert tr[0][1] == 0.0 and all(t1 >= t0 >= 0.0 for _, t0, t1, _ in tr)
    for name, (n, ms) in agg.items():
        mine = [t1 - t0 for nm, t0, t1, _ in tr if nm == name]
        assert len(mine) == n and abs(sum(mine) - ms) <= 1e-3 * max(ms, 1.0)
    assert all(crit for nm, _, _, crit in tr if nm == "chol_potrf_diag")
    assert not any(crit for nm, _, _, crit in tr if nm == "schur_gemm")
