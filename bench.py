#!/usr/bin/env python3
"""Benchmark: Newton steps/s and time-to-certificate of the Polya/SDP
interior-point method on one GB300.

Headline workload: the large system n=100, l=3, d_p=2, d1=d2=4 (K=30300 dual
variables, 28 + 36 blocks of 100 x 100), s=0.3, seed 0 of the synthetic
generator, in FP64: every result FP64-accurate, the two large contractions
(Schur complement, Cholesky trailing updates) by the Ozaki scheme on the BF16
tensor cores.  One "step" is one full predictor-corrector Newton step (Schur
assembly, dense Cholesky, both solves, directions, step length, update,
scalars) from the cold start X = Z = I, y = 0, restored (untimed) before every
timed step; the 7.3 GB Schur complement is rewritten every step (inputs far
larger than L2), and a 256 MB L2 flush precedes each step as well.

Also reported: the same step with FP64 FMA only (DFMA), the mixed-precision
form (steps/s, time-to-certificate, speedup over the measured FP64
time-to-certificate), the mid workload (n=20, l=4, d_p=2, d1=3, K=2100) in
FP64 as a second record, the oracle on a bounded sample of the headline
workload on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched under torchrun) every rank solves its own instance
(seed = rank): replicas, weak scaling, no collective on the data path.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="large", n=100, l=3, d_p=2, d1=4, s=0.3, seed=0)
MID = dict(name="mid", n=20, l=4, d_p=2, d1=3, s=0.3, seed=0)
METRIC = "Newton steps/s at FP64 accuracy (time-to-certificate in e2e; mixed-precision speedup in mixed)"
UNIT = "steps/s"
NOMINAL_BF16_TFLOPS = 2250.0
NOMINAL_TF32_TFLOPS = 1100.0
# BF16 slice products per FP64 multiply-add in the Ozaki scheme (8 slices, levels <= 9)
OZ_PAIRS = 36
OZ_DEPTH = 384
OZ_KERNEL = "k_ozaki_gemm_persist<64, 16>"
# DRAM bytes per updated element of OZ_KERNEL's lower trailing update at depth 384:
# dram__bytes_read.sum + dram__bytes_write.sum = 618.9 MB of one ncu capture of the
# 8192 x 8192 update (33.56 M elements; profiles/ozaki_gemm_persist_8192.md).  The C
# read-modify-write (16 B an element) dominates, so the traffic of a launch grows
# with the elements it updates; re-capture when the kernel changes.
OZ_DRAM_BYTES_PER_ELEMENT = 618.9e6 / (8192 * 8193 / 2)
KERNEL_OF = {"schur_gemm": "k_gemm_tn", "chol_syrk_gemm": "k_syrk_tri_persist", "oz_chol": OZ_KERNEL,
             "oz_schur": OZ_KERNEL, "chol32_syrk_tc": "k_tc_gemm_persist"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-samples", type=int, default=2, help="oracle samples of the headline step on the host")
    ap.add_argument("--mixed", type=int, default=1, help="also measure the mixed-precision path")
    ap.add_argument("--mixed-steps", type=int, default=5)
    ap.add_argument("--dfma", type=int, default=1, help="time one FP64-FMA-only step of the headline workload")
    ap.add_argument("--mid", type=int, default=1, help="also measure the mid workload in FP64")
    ap.add_argument("--mid-steps", type=int, default=30)
    ap.add_argument("--batch", type=int, default=64, help="instances of the batched-vs-sequential record (0: skip)")
    ap.add_argument("--mixed-workloads", default="mid,large")
    ap.add_argument("--extra-items", default="err,ex2,syrk,batch,warm")
    ap.add_argument("--err-large", type=int, default=1, help="also solve the large workload in plain FP64")
    ap.add_argument("--syrk-m", type=int, default=15000)
    ap.add_argument("--extra", action="store_true", help="measure the batched and warm-start rows instead")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--warm-train", type=int, default=1024)
    ap.add_argument("--warm-test", type=int, default=64)
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class NvmlSampler:
    """SM clock, power and clock-event reasons read through NVML (read-only
    queries) every 10 ms on a thread; selects the GPU by its PCI bus id."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, device: int):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(device)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(self.h)) == 0
        except Exception:
            ok = False
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.reasons_fn = fn
        mx = ctypes.c_uint()
        self.max_mhz = mx.value if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0 else None
        self.rows = []
        self.stop = threading.Event()

    def _poll(self):
        ct = self.ct
        mhz, mw, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        while not self.stop.is_set():
            a = self.lib.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz))
            b = self.lib.nvmlDeviceGetPowerUsage(self.h, ct.byref(mw))
            c = self.reasons_fn(self.h, ct.byref(rs))
            if a == 0:
                self.rows.append((mhz.value, mw.value / 1000.0 if b == 0 else None, rs.value if c == 0 else 0))
            time.sleep(0.01)

    def __enter__(self):
        self.t = threading.Thread(target=self._poll, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *exc):
        self.stop.set()
        self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "source": "nvml"}
        sm = [r[0] for r in self.rows]
        pw = [r[1] for r in self.rows if r[1] is not None]
        reasons = sorted({name for r in self.rows for bit, name in self.REASONS.items() if r[2] & bit})
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": self.max_mhz,
                "power_w_median": statistics.median(pw) if pw else None, "reasons": reasons,
                "samples": len(self.rows), "source": "nvml, 10 ms"}


class ClockSampler:
    """Clocks and throttle reasons during a timed region: NVML when it loads,
    else nvidia-smi every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None
        self.nvml = None

    def __enter__(self):
        try:
            self.nvml = NvmlSampler(self.device).__enter__()
            return self
        except Exception:
            self.nvml = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.nvml:
            self.nvml.__exit__(*exc)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.nvml:
            return self.nvml.summary()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "source": "nvidia-smi, 200 ms"}


def chol_flops(K, nb):
    """Algorithmic flops of one FP64 Cholesky by kernel: panel solves, updates of
    the next panel's rows (upper part only) and bulk trailing updates."""
    out = {"trsm": 0.0, "next": 0.0, "bulk": 0.0}
    for j0 in range(0, K, nb):
        wd = min(nb, K - j0)
        rest = K - j0 - wd
        if rest <= 0:
            break
        w2 = min(nb, rest)
        out["trsm"] += 2.0 * rest * wd * wd
        out["next"] += 2.0 * wd * (w2 * rest - w2 * (w2 - 1) / 2)
        r = rest - w2
        out["bulk"] += float(r) * (r + 1) * wd
    return out


def oz_outer(K):
    """Outer panel width of the Ozaki Cholesky: one 384-deep exact window from
    K = 8192 on, 256 below."""
    return OZ_DEPTH if K >= 8192 else 256


def chol_flops_ozaki(K, nb=32, ob=None):
    """Algorithmic flops of one FP64 Cholesky with Ozaki-scheme trailing updates, by
    kernel: 32-column panel solves (trsm), updates of the remaining columns of the
    inner panel's 128-column block (inner; of the whole outer panel below K = 8192),
    the block's update of the outer panel's columns right of it (block), the
    outer-panel-deep update of the next outer panel's columns (next) and of the
    rest of the trailing matrix (bulk), lower parts."""
    ob = ob or oz_outer(K)
    out = {"trsm": 0.0, "inner": 0.0, "block": 0.0, "next": 0.0, "bulk": 0.0}
    tri = lambda rows, cols: cols * rows - cols * (cols - 1) / 2      # lower part of a rows x cols block
    for J0 in range(0, K, ob):
        wo = min(ob, K - J0)
        bw = 128 if K >= 8192 else wo
        for b0 in range(J0, J0 + wo, bw):
            wb = min(bw, J0 + wo - b0)
            for j0 in range(b0, b0 + wb, nb):
                w = min(nb, K - j0)
                rest = K - j0 - w
                if rest <= 0:
                    break
                out["trsm"] += 2.0 * rest * w * w
                nrem = b0 + wb - (j0 + w)
                if nrem > 0:
                    out["inner"] += 2.0 * w * tri(rest, nrem)
            nrem_o, rest_b = J0 + wo - (b0 + wb), K - (b0 + wb)
            if nrem_o > 0 and rest_b > 0:
                out["block"] += 2.0 * wb * tri(rest_b, nrem_o)
        r = K - (J0 + wo)
        if r <= 0:
            break
        w2 = min(ob, r)
        out["next"] += 2.0 * wo * tri(r, w2)
        m = r - w2
        out["bulk"] += float(m) * (m + 1) * wo
    return out


def oracle_steps(A, w, nsteps):
    """Time nsteps oracle Newton steps from the cold start (test infrastructure)."""
    from oracle import ipm, sdp
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    times = []
    for _ in range(nsteps):
        st = ipm.start_point(prob)
        t0 = time.perf_counter()
        ipm.newton_step(prob, st, ipm.Options())
        times.append(time.perf_counter() - t0)
    return times


def oracle_sample(A, w, blocks=((0, 0),)):
    """A bounded sample of one oracle Newton step of workload w on the host
    cores: the oracle's Schur complement restricted to the (a, b) blocks listed
    (of L0^2, at the cold start X = Z = I) and its dense Cholesky (numpy) on an
    SPD matrix of order K/4.  The step time is estimated as L0^2 / len(blocks)
    times the first plus 64 times the second (cubic work); the step's remaining
    parts (operators, block inverses, step length) are left out, so the estimate
    is a lower bound.  Returns (estimated step seconds, seconds spent)."""
    from oracle import sdp
    prob = sdp.Problem(A, w["d_p"], w["d1"])
    I = prob.identity_blocks()
    k4 = max(1, prob.K // 4)
    rng = np.random.default_rng(0)
    R = rng.random((k4, k4))
    S = R + R.T + (2.0 * k4 + 1.0) * np.eye(k4)       # diagonally dominant, SPD
    t0 = time.perf_counter()
    prob.schur_structured(I, I, blocks=list(blocks))
    t1 = time.perf_counter()
    np.linalg.cholesky(S)
    t2 = time.perf_counter()
    est = prob.L0 ** 2 / len(blocks) * (t1 - t0) + 64.0 * (t2 - t1)
    return est, t2 - t0


def chol32_bulk_flops(K, nb=128, outer=4):
    """Useful flops of the mixed form's outer trailing updates (the persistent
    3xTF32 kernel on the main stream), lower triangle: per outer panel of
    wo = outer*nb columns, m(m+1) wo with m the rows below the next outer panel."""
    ob = outer * nb
    tot, launches = 0.0, 0
    for J0 in range(0, K, ob):
        wo = min(ob, K - J0)
        rest = K - (J0 + wo)
        if rest <= 0:
            break
        m = rest - min(ob, rest)
        if m > 0:
            tot += float(m) * (m + 1) * wo
            launches += 1
    return tot, launches


def measure_mixed(bd, synth, name, device, nsteps, crit_sms=0):
    """Mixed-precision Newton steps/s (from the cold start, CUDA events around
    each step on the library's stream) and the full time-to-certificate."""
    import torch
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    stream = torch.cuda.Stream()
    opts = bd.psdp_default_opts(stream=stream.cuda_stream, device=device, precision=1, crit_sms=crit_sms)
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A, opts)
    try:
        X0, Z0, y0 = bd.psdp_get_iterate(h)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        ms = []
        fallback = 0.0
        with ClockSampler(device) as clk:
            for i in range(nsteps + 1):
                bd.psdp_load_iterate(h, X0, Z0, y0)
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s, info = bd.psdp_step(h)
                e1.record(stream)
                torch.cuda.synchronize()
                if s != 0:
                    raise RuntimeError(f"mixed step: {bd.STATUS[s]}")
                fallback = max(fallback, info[13])
                if i > 0:                      # the first step captures the graph
                    ms.append(e0.elapsed_time(e1))
        work = bd.psdp_work(h)
        # per-kernel breakdown from CUDA events inside the (re-captured) step graph
        bd.psdp_profile_enable(h, True)
        bd.psdp_load_iterate(h, X0, Z0, y0)
        bd.psdp_step(h)
        bd.psdp_profile_reset(h)
        bd.psdp_load_iterate(h, X0, Z0, y0)
        bd.psdp_step(h)
        prof = bd.psdp_profile_get(h)
        bd.psdp_profile_enable(h, False)
    finally:
        bd.psdp_destroy(h)
    t0 = time.perf_counter()
    with bd.Solver(A, w["d_p"], w["d1"], device=device, precision=1, crit_sms=crit_sms) as s:
        status, iters, info = s.solve()
        verdict, _, _ = s.certify()
        bd.psdp_get_P(s.h)
    t1 = time.perf_counter()
    roof = None
    if "chol32_syrk_tc" in prof and prof["chol32_syrk_tc"][0] > 0:
        pk, pk_kind = peaks()
        tf32_peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * NOMINAL_TF32_TFLOPS / NOMINAL_BF16_TFLOPS
        useful, nl = chol32_bulk_flops(polya_K(w), work["nb_chol32"])
        launches, tms = prof["chol32_syrk_tc"]
        issued = 3.0 * useful / max(nl, 1)          # 3xTF32: three TF32 products per useful one
        ach = issued / (tms / launches * 1e-3) / 1e12
        roof = {"kernel": "k_tc_gemm_persist (chol32_syrk_tc, 3xTF32 trailing update)", "bound": "tensor",
                "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak,
                "useful_tflops": useful / max(nl, 1) / (tms / launches * 1e-3) / 1e12,
                "share_of_step": tms / sum(v[1] for v in prof.values()),
                "peak_source": f"{pk_kind} bf16 sustained x nominal TF32/BF16 {NOMINAL_TF32_TFLOPS:.0f}/{NOMINAL_BF16_TFLOPS:.0f}",
                "traffic": None}
    return {"workload": f"n={w['n']} l={w['l']} d_p={w['d_p']} d1=d2={w['d1']} s={w['s']} seed=0",
            "roofline": roof,
            "ms_per_step": sum(ms) / len(ms), "steps_per_s": 1e3 * len(ms) / sum(ms),
            "time_to_certificate_s": t1 - t0, "newton_steps": iters, "status": status, "verdict": verdict,
            "relgap": info["relgap"], "fp64_fallback": bool(info["fallback"] or fallback),
            "pcg_iterations_last_step": info["refine_sweeps"], "schur_flops_per_step": work["schur_flops"],
            "chol_flops_per_step": work["chol_flops"], "clocks": clk.summary(),
            "kernels_ms_per_step": {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in prof.items()}}


def measure_fp64_step(bd, synth, name, device):
    """One plain FP64 Newton step of a workload from the cold start (CUDA events
    on the library's stream; the step is also the graph capture, a few ms of
    host work against seconds of device work at the large size)."""
    import torch
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    stream = torch.cuda.Stream()
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A,
                      bd.psdp_default_opts(stream=stream.cuda_stream, device=device, precision=0))
    try:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s, info = bd.psdp_step(h)
        e1.record(stream)
        torch.cuda.synchronize()
        if s != 0:
            raise RuntimeError(f"fp64 step: {bd.STATUS[s]}")
        return e0.elapsed_time(e1)
    finally:
        bd.psdp_destroy(h)


def measure_batch(bd, synth, count, device, n_range=(8, 48), precision=1):
    """Uneven instances drawn like the batched workload (n ~ U{8..48}, l ~ U{2,3,4},
    d_p ~ U{1,2}, d1 ~ U{1..4}, s ~ U[0.05, 3]) solved together in one batch graph
    per iteration; set-up, solve and certificates all timed."""
    inst = synth.batch_instances(count, base_seed=1000, n_range=n_range)
    t0 = time.perf_counter()
    hs = [bd.psdp_setup(d["n"], d["l"], d["d_p"], d["d1"], d["A"],
                        bd.psdp_default_opts(precision=precision, device=device)) for d in inst]
    t1 = time.perf_counter()
    try:
        status, iters = bd.psdp_solve_batch(hs)
        t2 = time.perf_counter()
        verdicts = [bd.psdp_certify(h)[0] for h in hs]
        t3 = time.perf_counter()
    finally:
        for h in hs:
            bd.psdp_destroy(h)
    Ks = [polya_K(d) for d in inst]
    return {"instances": count, "n_range": list(n_range), "precision": "mixed" if precision else "fp64",
            "newton_steps_total": int(sum(iters)), "steps_per_s": sum(iters) / (t2 - t1),
            "setup_s": t1 - t0, "solve_s": t2 - t1, "certify_s": t3 - t2, "time_to_all_certificates_s": t3 - t0,
            "certified": int(sum(verdicts)), "status_counts": {s: status.count(s) for s in sorted(set(status))},
            "K_max": max(Ks), "K_mean": float(np.mean(Ks))}


def measure_batch_vs_sequential(bd, synth, count, device, precision=0):
    """The same uneven instances (the batch workload's draw: n ~ U{8..48}, l ~
    U{2,3,4}, d_p ~ U{1,2}, d1 ~ U{1..4}, s ~ U[0.05, 3]) solved together
    (psdp_solve_batch: one graph launch per interior-point iteration over every
    unfinished instance) and one after another (psdp_solve each), set-up and
    certificates included on both sides; statuses and iteration counts must agree."""
    inst = synth.batch_instances(count, base_seed=1000)

    def setup_all():
        return [bd.psdp_setup(d["n"], d["l"], d["d_p"], d["d1"], d["A"],
                              bd.psdp_default_opts(precision=precision, device=device)) for d in inst]

    t0 = time.perf_counter()
    hs = setup_all()
    try:
        st_b, it_b = bd.psdp_solve_batch(hs)
        v_b = [bd.psdp_certify(h)[0] for h in hs]
    finally:
        for h in hs:
            bd.psdp_destroy(h)
    t1 = time.perf_counter()
    st_s, it_s, v_s = [], [], []
    for d in inst:
        h = bd.psdp_setup(d["n"], d["l"], d["d_p"], d["d1"], d["A"],
                          bd.psdp_default_opts(precision=precision, device=device))
        try:
            s, it, _ = bd.psdp_solve(h)
            st_s.append(bd.STATUS[s])
            it_s.append(it)
            v_s.append(bd.psdp_certify(h)[0])
        finally:
            bd.psdp_destroy(h)
    t2 = time.perf_counter()
    steps = int(sum(it_b))
    return {"instances": count, "precision": "mixed" if precision else "fp64",
            "K_max": max(polya_K(d) for d in inst), "newton_steps": steps,
            "batched_s": t1 - t0, "sequential_s": t2 - t1, "batched_steps_per_s": steps / (t1 - t0),
            "sequential_steps_per_s": int(sum(it_s)) / (t2 - t1), "speedup": (t2 - t1) / (t1 - t0),
            "same_outcomes": list(st_b) == st_s and list(it_b) == it_s and v_b == v_s,
            "certified": int(sum(v_b)), "status_counts": {s: list(st_b).count(s) for s in sorted(set(st_b))}}


def polya_K(d):
    from math import comb
    return comb(d["d_p"] + d["l"] - 1, d["l"] - 1) * d["n"] * (d["n"] + 1) // 2


def measure_warm(bd, n_train, n_test, device):
    """Learned warm start on the n=32, l=3, d_p=2, d1=3 family, s ~ U[0.1, 1.5]."""
    from paper_1411_3769_gb300 import warmstart as ws
    n, l, d_p, d1 = 32, 3, 2, 3
    t0 = time.perf_counter()
    train_sys = ws.draw(n_train, n, l, (0.1, 1.5), base_seed=5000)
    test_sys = ws.draw(n_test, n, l, (0.1, 1.5), base_seed=9000)
    F, T, status, iters, verdicts = ws.solve_family(train_sys, d_p, d1, stop_iter=ws.K_TARGET)
    t1 = time.perf_counter()
    ok = np.array([s in ("OK", "EMAXITER") for s in status])
    m, loss = ws.train(F[ok], T[ok], width=1024, epochs=200, batch=64, lr=1e-3)
    t2 = time.perf_counter()
    try:
        res = ws.evaluate(m, test_sys, d_p, d1)
        # held-out prediction error (standardised by the training targets) of the
        # network and of the training-target mean
        mean = T[ok].mean(axis=0)
        sd = np.maximum(T[ok].std(axis=0), 1e-6)
        Fte, Tte, st_te, _, _ = ws.solve_family(test_sys, d_p, d1, stop_iter=ws.K_TARGET)
        okt = np.array([s in ("OK", "EMAXITER") for s in st_te])
        P = bd.psdp_mlp_predict(m, Fte[okt], T.shape[1])
        res["heldout_std_mse"] = {"network": float((((P - Tte[okt]) / sd) ** 2).mean()),
                                  "mean_predictor": float((((mean - Tte[okt]) / sd) ** 2).mean())}
        # ablation: the same warm-start machinery fed the training-target mean
        abl = ws.evaluate(None, test_sys, d_p, d1, predict=lambda f, k: np.tile(mean, (f.shape[0], 1)))
        res["mean_predictor"] = {"warm_iters": abl["warm_iters"], "iterations_saved": abl["iterations_saved"],
                                 "verdicts_agree": abl["verdicts_agree"], "fallbacks": abl["fallbacks"]}
        # the same held-out systems solved in plain FP64 from the cold start: the
        # mixed + learned-warm-start form against the plain GPU path, same stopping rule
        f64 = ws.cold_solves(test_sys, d_p, d1, precision=0)
        res["fp64_cold"] = {"seconds": f64["seconds"], "iters": f64["iters"]}
        res["mixed_warm_vs_fp64_cold"] = {
            "speedup_time_to_certificate": f64["seconds"] / res["warm_s"],
            "mixed_cold_speedup": f64["seconds"] / res["cold_s"],
            "verdicts_agree": bool(all(a == b for a, b in zip(f64["verdicts"], res["warm_verdicts"])))}
        res.pop("warm_verdicts", None)
    finally:
        bd.psdp_mlp_destroy(m)
    res.update(train_instances=int(ok.sum()), train_generate_s=t1 - t0, train_s=t2 - t1, final_train_loss=loss,
               family="n=32 l=3 d_p=2 d1=d2=3 s~U[0.1,1.5]")
    return res


def measure_syrk_probe(bd, M, K=128, ctas=152):
    """The persistent 3xTF32 trailing update alone on an M x M lower-triangular
    update of depth K (the shape of one FP32 Cholesky panel update), random
    operands; CUDA events around the launch."""
    rng = np.random.default_rng(3)
    P = rng.standard_normal((M, K)).astype(np.float32)
    C0 = np.zeros((M, M), dtype=np.float32)
    _, ms = bd.psdp_tc_gemm_persist_check(P, P, C0, split=3, tri=1, ctas=ctas, timing=True)
    T = (M + 127) // 128
    tiles = T * (T + 1) // 2
    c_bytes = tiles * 128 * 128 * 4 * 2            # C read + write per tile
    flops = tiles * 2.0 * 128 * 128 * K            # useful product (the 3xTF32 split issues 3x)
    return {"M": M, "K": K, "ctas": ctas, "tiles": tiles, "ms": ms, "c_traffic_gbs": c_bytes / (ms * 1e-3) / 1e9,
            "useful_tflops": flops / (ms * 1e-3) / 1e12}


def load_example2():
    """The six 3x3 coefficients printed in Sec. V, Example 2 (exponent -> matrix)."""
    mats, cur = {}, None
    with open(os.path.join(ROOT, "tests", "golden", "example2_A.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("A"):
                cur = tuple(int(x) for x in line.split()[1:])
                mats[cur] = []
            else:
                mats[cur].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


def measure_example2(degrees=((1, 1), (2, 2), (2, 3), (3, 3), (3, 4))):
    """Upper bounds on L_opt = -0.111 (Sec. V, Example 2) by batched multisection
    (7 scales per round, 4 rounds, scale range [-0.2, 1]), wall time per bound."""
    from paper_1411_3769_gb300 import robust
    terms = load_example2()
    out = []
    for d_p, d1 in degrees:
        t0 = time.perf_counter()
        bound, trace = robust.multisection(terms, -0.2, 1.0, d_p, d1, points=7, rounds=4)
        out.append({"d_p": d_p, "d1=d2": d1, "bound": bound, "solves": len(trace),
                    "seconds": time.perf_counter() - t0})
    return {"L_opt_printed": -0.111, "bounds": out}


def measure_mixed_error(bd, synth, name, device, with_oracle):
    """The mixed-precision solution against the plain FP64 GPU solution (and the
    FP64 oracle where it finishes): optimal value a^T y, P_h, verdicts."""
    w = synth.WORKLOADS[name]
    A = synth.system(w["n"], w["l"], w["s"], 0)
    res = {}
    for prec in (0, 1):
        t0 = time.perf_counter()
        with bd.Solver(A, w["d_p"], w["d1"], device=device, precision=prec) as s:
            status, iters, info = s.solve()
            verdict = s.certify()[0]
            P = bd.psdp_get_P(s.h)
        res[prec] = dict(status=status, iters=iters, psi=info["psi"], relgap=info["relgap"], verdict=verdict, P=P,
                         seconds=time.perf_counter() - t0)
    out = {"workload": name, "fp64": {k: v for k, v in res[0].items() if k != "P"},
           "mixed": {k: v for k, v in res[1].items() if k != "P"},
           "psi_rel_err_vs_fp64_gpu": abs(res[1]["psi"] - res[0]["psi"]) / abs(res[0]["psi"]),
           "P_max_rel_diff_vs_fp64_gpu": float(np.abs(res[1]["P"] - res[0]["P"]).max() / np.abs(res[0]["P"]).max())}
    if with_oracle:
        from oracle import certify, ipm, sdp
        t0 = time.perf_counter()
        prob = sdp.Problem(A, w["d_p"], w["d1"])
        st, state = ipm.solve(prob, ipm.Options())
        psi_o = float(prob.a @ state.y)
        Po = prob.P_from_y(state.y)
        out["oracle"] = {"status": st, "iters": state.it, "psi": psi_o,
                         "verdict": certify.certify(prob, state.y)["verdict"], "seconds": time.perf_counter() - t0}
        out["psi_rel_err_vs_oracle"] = {"mixed": abs(res[1]["psi"] - psi_o) / abs(psi_o),
                                        "fp64": abs(res[0]["psi"] - psi_o) / abs(psi_o)}
        out["P_max_rel_diff_vs_oracle"] = {"mixed": float(np.abs(res[1]["P"] - Po).max() / np.abs(Po).max()),
                                           "fp64": float(np.abs(res[0]["P"] - Po).max() / np.abs(Po).max())}
    return out


def run_extra(args):
    """Batched, learned-warm-start and kernel-probe rows (minutes of GPU time;
    not the default line)."""
    import torch
    torch.cuda.set_device(0)
    from paper_1411_3769_gb300 import build
    build.build()
    from paper_1411_3769_gb300 import binding as bd
    from paper_1411_3769_gb300 import synth
    items = [x for x in args.extra_items.split(",") if x]
    out = {}
    if "err" in items:
        out["mixed_error"] = [measure_mixed_error(bd, synth, "mid", 0, True)]
        if args.err_large:
            out["mixed_error"].append(measure_mixed_error(bd, synth, "large", 0, False))
    if "ex2" in items:
        out["example2"] = measure_example2()
    if "syrk" in items:
        out["syrk_probe"] = [measure_syrk_probe(bd, args.syrk_m, ctas=c) for c in (152, 136)]
    if "batch" in items:
        out["batch"] = measure_batch(bd, synth, args.batch_count, 0)
    if "warm" in items:
        out["warm_start"] = measure_warm(bd, args.warm_train, args.warm_test, 0)
    print(json.dumps(out), flush=True)


def run_reference(args):
    """The oracle (the paper ships no code) on the headline workload: each step
    is one bounded sample of an oracle Newton step (oracle_sample), the step
    time estimated from it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1411_3769_gb300 import synth
    w = WORKLOAD
    A = synth.system(w["n"], w["l"], w["s"], w["seed"])
    warm = max(1, args.warmup)
    for _ in range(warm):                             # untimed warm-up samples (~6 s each)
        oracle_sample(A, w)
    est = [oracle_sample(A, w)[0] for _ in range(args.steps)]
    tot = sum(est)
    v = args.steps / tot
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": warm, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} samples of one oracle Newton step at the cold start, each: the "
                                       "Schur complement's (0,0) block of 36 and a numpy Cholesky of order K/4, "
                                       "scaled to a step (x36, x64); the step's other parts left out"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(w):
    K = polya_K(w)
    return {"workload": f"n={w['n']} l={w['l']} d_p={w['d_p']} d1=d2={w['d1']} (K={K}) s={w['s']} seed={w['seed']}",
            "precision": "FP64 results", "l2": "Schur complement of 8K^2 bytes rewritten every step, plus a 256 MB flush"}


def time_steps(bd, torch, h, stream, X0, Z0, y0, flush, nsteps):
    """nsteps Newton steps from the restored cold start, each bracketed by CUDA
    events on the library's stream after an L2 flush on it; returns ms per step."""
    evs = []
    for _ in range(nsteps):
        bd.psdp_load_iterate(h, X0, Z0, y0)
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s, info = bd.psdp_step(h)
        if s != 0:
            raise RuntimeError(f"psdp_step failed: {bd.STATUS[s]}")
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def profile_step(bd, torch, h, stream, X0, Z0, y0, flush, nsteps=1):
    """Per-kernel CUDA-event durations inside the re-captured step graph."""
    bd.psdp_profile_enable(h, True)
    time_steps(bd, torch, h, stream, X0, Z0, y0, flush, 1)
    bd.psdp_profile_reset(h)
    ms = time_steps(bd, torch, h, stream, X0, Z0, y0, flush, nsteps)
    prof = bd.psdp_profile_get(h)
    bd.psdp_profile_enable(h, False)
    return prof, sum(ms)


def time_to_certificate(bd, A, w, local, **opts):
    """setup + solve + certify + P readback through the C ABI with host buffers."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with bd.Solver(A, w["d_p"], w["d1"], device=local, **opts) as s:
        status, iters, info = s.solve()
        verdict, _, _ = s.certify()
        P = bd.psdp_get_P(s.h)
        y = bd.psdp_get_y(s.h)
    t = time.perf_counter() - t0
    return {"seconds": t, "newton_steps": iters, "status": status, "verdict": verdict, "relgap": info["relgap"],
            "psi": info["psi"], "P_bytes": P.nbytes, "y": y}


def fp64_roofline(kern, prof, prof_ms, steps, K, work, engines, fp64_peak, pk, pk_kind):
    """Per-kernel algorithmic rates of the FP64 step and the dominant contraction's
    roofline.  Ozaki kernels are bound by the BF16 tensor pipe: their achieved rate
    counts the 36 exact BF16 slice products each FP64 multiply-add takes."""
    oz_c, oz_s = engines["cholesky"] == "ozaki", engines["schur"] == "ozaki"
    cf = chol_flops_ozaki(K) if oz_c else chol_flops(K, work["nb_chol"])
    for name, fl in (("schur_gemm", work["schur_flops"]), ("chol_syrk_gemm", cf["bulk"]),
                     ("chol_syrk_next", cf["next"]), ("chol_trsm_gemm", cf["trsm"]),
                     ("chol_inner_update", cf.get("inner", 0.0)), ("chol_block_update", cf.get("block", 0.0))):
        if name in prof and prof[name][0] > 0:
            launches, tms = prof[name]
            per_step = launches / steps
            avg = tms / launches
            kern[name] = {"launches_per_step": per_step, "avg_ms": avg,
                          "fp64_tflops": fl / per_step / (avg * 1e-3) / 1e12, "share_of_step": tms / prof_ms}
    for name in ("chol_potrf_diag", "dense_solve", "schur_operands", "schur_gather", "schur_oz_split", "chol_oz_split",
                 "block_chol_inv", "block_maxstep"):
        if name in prof and prof[name][0] > 0:
            kern[name] = {"launches_per_step": prof[name][0] / steps, "avg_ms": prof[name][1] / prof[name][0],
                          "share_of_step": prof[name][1] / prof_ms}
    dom = max(("schur_gemm", "chol_syrk_gemm"), key=lambda k: kern.get(k, {}).get("share_of_step", 0))
    rate = kern.get(dom, {}).get("fp64_tflops")
    ozaki = oz_c if dom == "chol_syrk_gemm" else oz_s
    if ozaki:
        peak = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        ach = OZ_PAIRS * rate if rate else None
        roof = {"kernel": OZ_KERNEL + " (" + dom + ", FP64 by the Ozaki scheme)", "bound": "tensor", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": (ach / peak) if ach else None,
                "peak_source": f"{pk_kind} bf16 sustained (kernel timed inside a seconds-long step)",
                "counted": f"{OZ_PAIRS} BF16 slice products per FP64 multiply-add of the algorithmic work",
                "fp64_equivalent_tflops": rate, "fp64_measured_peak_tflops": fp64_peak,
                "fp64_equivalent_over_fp64_peak": (rate / fp64_peak) if rate else None}
    else:
        roof = {"kernel": KERNEL_OF[dom] + " (" + dom + ")", "bound": "fp64", "achieved": rate, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": (rate / fp64_peak) if rate else None,
                "peak_source": "measured: the larger of the DFMA and DMMA probes (psdp_fp64_peaks)"}
    roof["traffic"] = None
    if ozaki and dom == "chol_syrk_gemm" and dom in kern:
        # elements one bulk launch updates: its flops / (2 x depth), on average
        elems = cf["bulk"] / (2.0 * oz_outer(K)) / kern[dom]["launches_per_step"]
        roof["traffic"] = OZ_DRAM_BYTES_PER_ELEMENT * elems
        roof["traffic_unit"] = "bytes per launch"
        roof["traffic_source"] = (f"ncu capture of {OZ_KERNEL} on the 8192 x 8192 lower update at depth 384: "
                                  f"{OZ_DRAM_BYTES_PER_ELEMENT:.2f} B per updated element, times the elements of "
                                  "an average bulk launch")
        roof["algorithmic_bytes"] = 16.0 * elems      # C read and written once
    return roof


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1411_3769_gb300 import build
    build.build()
    from paper_1411_3769_gb300 import binding as bd
    from paper_1411_3769_gb300 import synth

    pk, pk_kind = peaks()
    dfma_peak, dmma_peak = bd.psdp_fp64_peaks(local)
    fp64_peak = max(dfma_peak, dmma_peak)
    w = WORKLOAD
    A = synth.system(w["n"], w["l"], w["s"], w["seed"] + rank)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    h = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A, bd.psdp_default_opts(stream=stream.cuda_stream,
                                                                                  device=local))
    engines = bd.psdp_engines(h)
    X0, Z0, y0 = bd.psdp_get_iterate(h)
    time_steps(bd, torch, h, stream, X0, Z0, y0, flush, max(args.warmup, 3))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = time_steps(bd, torch, h, stream, X0, Z0, y0, flush, args.steps)
    tot_ms = sum(ms)
    y_step = bd.psdp_get_y(h)                          # one step from the cold start
    work = bd.psdp_work(h)
    sizes = bd.psdp_sizes(h)
    # per-kernel durations from a second, profiled region (events slow the step)
    prof, prof_ms = profile_step(bd, torch, h, stream, X0, Z0, y0, flush, 1)
    bd.psdp_destroy(h)
    if dist:
        from paper_1411_3769_gb300 import replicas
        tot_ms = replicas.max_over_ranks(tot_ms, dist, device="cuda")    # the slowest replica
        dist.barrier()
    ttc = time_to_certificate(bd, A, w, local)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    kern = {"_profiled_ms_per_step": prof_ms}
    roof = fp64_roofline(kern, prof, prof_ms, 1, sizes["K"], work, engines, fp64_peak, pk, pk_kind)

    # ---- the same step with FP64 FMA only, for the speedup and the parity of the two engines
    dfma = {}
    if args.dfma:
        st2 = torch.cuda.Stream()
        h2 = bd.psdp_setup(w["n"], w["l"], w["d_p"], w["d1"], A,
                           bd.psdp_default_opts(stream=st2.cuda_stream, device=local, fp64_gemm=1))
        try:
            m2 = time_steps(bd, torch, h2, st2, X0, Z0, y0, flush, 1)
            y2 = bd.psdp_get_y(h2)
            dfma = {"ms_per_step": m2[0], "speedup_of_headline_step": m2[0] / (tot_ms / args.steps),
                    "y_rel_diff_vs_headline_step": float(np.abs(y_step - y2).max() / np.abs(y2).max())}
        finally:
            bd.psdp_destroy(h2)

    # ---- mixed precision (3xTF32 tensor cores + FP64 PCG)
    mixed = {}
    if args.mixed:
        for wl in [x for x in args.mixed_workloads.split(",") if x]:
            try:
                mixed[wl] = measure_mixed(bd, synth, wl, local, args.mixed_steps)
            except Exception as exc:   # report, do not lose the main line
                mixed[wl] = {"error": str(exc)[:200]}
        lg = mixed.get("large", {})
        if "time_to_certificate_s" in lg:
            lg["fp64_time_to_certificate_s"] = ttc["seconds"]
            lg["speedup_time_to_certificate_vs_fp64"] = ttc["seconds"] / lg["time_to_certificate_s"]
            lg["speedup_step_vs_fp64"] = (tot_ms / args.steps) / lg["ms_per_step"]
            if dfma:
                lg["speedup_step_vs_dfma_fp64"] = dfma["ms_per_step"] / lg["ms_per_step"]

    # ---- the mid workload in FP64 (second record)
    mid = {}
    if args.mid:
        wm = MID
        Am = synth.system(wm["n"], wm["l"], wm["s"], wm["seed"])
        hm = bd.psdp_setup(wm["n"], wm["l"], wm["d_p"], wm["d1"], Am,
                           bd.psdp_default_opts(stream=stream.cuda_stream, device=local))
        try:
            Xm, Zm, ym = bd.psdp_get_iterate(hm)
            time_steps(bd, torch, hm, stream, Xm, Zm, ym, flush, 3)
            with ClockSampler(local) as clk_m:
                mm = time_steps(bd, torch, hm, stream, Xm, Zm, ym, flush, args.mid_steps)
            wk = bd.psdp_work(hm)
            eng_m = bd.psdp_engines(hm)
            pm, pm_ms = profile_step(bd, torch, hm, stream, Xm, Zm, ym, flush, 5)
        finally:
            bd.psdp_destroy(hm)
        km = {"_profiled_ms_per_step": pm_ms / 5}
        roof_m = fp64_roofline(km, pm, pm_ms, 5, polya_K(wm), wk, eng_m, fp64_peak, pk, pk_kind)
        tm = time_to_certificate(bd, Am, wm, local, eps=1e-8)
        mid = {"config": workload_config(wm), "engines": eng_m, "steps": args.mid_steps,
               "ms_per_step": sum(mm) / len(mm), "steps_per_s": 1e3 * len(mm) / sum(mm), "roofline": roof_m,
               "kernels": km, "clocks": clk_m.summary(),
               "time_to_certificate_eps_1e-8": {k: v for k, v in tm.items() if k != "y"}}

    # ---- many uneven instances: batched against one after another
    batch = {}
    if args.batch > 0:
        try:
            batch = measure_batch_vs_sequential(bd, synth, args.batch, local)
        except Exception as exc:
            batch = {"error": str(exc)[:200]}

    # ---- the oracle on a bounded sample of the headline workload
    est = [oracle_sample(A, w)[0] for _ in range(max(1, args.cpu_samples))]
    cpu = {"value": len(est) / sum(est), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"{len(est)} samples of one oracle Newton step at the cold start, each: the Schur complement's "
                     "(0,0) block of 36 and a numpy Cholesky of order K/4, scaled to a step (x36, x64); the "
                     "step's other parts left out (a lower bound on its time)"}

    value = world * args.steps / (tot_ms * 1e-3)
    iters = ttc["newton_steps"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(w), engines=engines,
                           parallelism="replicas" if world > 1 else "single"),
            "roofline": roof, "kernels": kern, "cpu_baseline": cpu,
            "e2e": {"value": (iters / ttc["seconds"]) if iters else None, "unit": UNIT,
                    "h2d_bytes_per_step": A.nbytes / max(iters, 1),
                    "d2h_bytes_per_step": (ttc["P_bytes"] + 16 * 8 * iters + 4 * iters) / max(iters, 1),
                    "time_to_certificate_s": ttc["seconds"], "newton_steps": iters, "status": ttc["status"],
                    "verdict": ttc["verdict"], "relgap": ttc["relgap"]},
            "fp64_dfma_step": dfma, "mixed": mixed, "mid_fp64": mid, "batch": batch,
            "fp64_peaks_tflops": {"dfma": dfma_peak, "dmma": dmma_peak},
            "gpu_launches": int(work["kernels_per_step"]) * args.steps,
            "clocks": clk.summary(),
            "work": {"schur_flops_per_step": work["schur_flops"], "chol_flops_per_step": work["chol_flops"],
                     "schur_terms": work["schur_terms"], "schur_dense_flops": work["schur_dense_flops"]}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.extra:
        run_extra(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
