"""Time Newton steps of one synthetic workload from its cold start.

    python -m paper_1411_3769_gb300.run_step --workload mid --precision fp64 --engine auto --steps 3

Every step starts from the cold-start iterate (restored untimed), so each
timed step does the same work; the time is the host wall time of psdp_step,
which returns after the step has finished on the device.  Prints one JSON
line: the workload, the FP64 engines, milliseconds per step and the kernels a
step launches.  Meant for profiling one configuration (the ncu summaries give
their commands in this form) and for quick timings of an engine choice.
"""

from __future__ import annotations

import argparse
import json
import time

from . import synth


def main(argv=None) -> dict:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="mid", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--engine", default="auto", choices=["auto", "fma", "ozaki"],
                    help="FP64 engine of the Schur contraction and the Cholesky updates")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)

    from . import build
    build.build()
    from . import binding as bd

    w = synth.WORKLOADS[args.workload]
    A = synth.system(w["n"], w["l"], w["s"], args.seed)
    opts = bd.psdp_default_opts(precision=0 if args.precision == "fp64" else 1,
                                fp64_gemm={"auto": 0, "fma": 1, "ozaki": 2}[args.engine])
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A, opts)
    try:
        X0, Z0, y0 = bd.psdp_get_iterate(h)
        ms = []
        for i in range(args.warmup + args.steps):
            bd.psdp_load_iterate(h, X0, Z0, y0)
            t0 = time.perf_counter()
            status, _ = bd.psdp_step(h)
            t1 = time.perf_counter()
            if status != 0:
                raise RuntimeError(f"psdp_step: {bd.STATUS.get(status, status)}")
            if i >= args.warmup:
                ms.append(1e3 * (t1 - t0))
        out = dict(workload=args.workload, precision=args.precision, engines=bd.psdp_engines(h),
                   ms_per_step=sum(ms) / max(len(ms), 1), ms=ms,
                   kernels_per_step=bd.psdp_work(h)["kernels_per_step"])
    finally:
        bd.psdp_destroy(h)
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
