"""Thin ctypes binding of ``include/polya_sdp.h`` (argument marshalling only).

Every function here has the name of the C entry point it wraps and does
nothing but convert numpy arrays to pointers and statuses to exceptions; all
computation happens in ``lib/libpolya_sdp.so``.  Loading fails loudly when the
library has not been built: there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpolya_sdp.so")

INFO_LEN = 16
INFO_FIELDS = ("phi", "psi", "relgap", "pres", "dres", "mu", "tp", "td", "trZX", "trX", "BXnorm",
               "iters", "refine_sweeps", "fallback", "r14", "r15")

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ECHOL_BLOCK", 5: "ECHOL_SCHUR", 6: "EMAXITER",
          7: "ESTEP", 8: "EUNBOUNDED", 9: "ENAN", 10: "ETIMEOUT", 11: "ESTATE"}

# every symbol the header declares
EXPORTS = ("psdp_default_opts", "psdp_setup", "psdp_sizes", "psdp_step", "psdp_solve", "psdp_certify",
           "psdp_grid_check", "psdp_get_P", "psdp_get_y", "psdp_get_tables", "psdp_load_iterate",
           "psdp_get_iterate", "psdp_get_schur", "psdp_get_schur_cols", "psdp_apply_BT", "psdp_apply_B", "psdp_profile_enable",
           "psdp_profile_reset", "psdp_profile_get", "psdp_profile_trace", "psdp_work", "psdp_stream", "psdp_fp64_peak",
           "psdp_destroy", "psdp_strerror", "psdp_tc_gemm_check", "psdp_tc_gemm_persist_check", "psdp_trsv_timeout_check", "psdp_get_schur_mixed",
           "psdp_tc_gemm_noalloc", "psdp_solve_batch", "psdp_autotune", "psdp_set_start", "psdp_mlp_create",
           "psdp_mlp_destroy", "psdp_mlp_params", "psdp_mlp_grads", "psdp_mlp_train", "psdp_mlp_predict",
           "psdp_fp64_peaks", "psdp_ozaki_gemm_check", "psdp_engines", "psdp_set_constant_term",
           "psdp_set_objective", "psdp_autotune_ex")


class Opts(C.Structure):
    _fields_ = [("delta", C.c_double), ("delta_L", C.c_double), ("eps", C.c_double), ("sigma", C.c_double),
                ("tau", C.c_double), ("max_iter", C.c_int), ("d2", C.c_int), ("d_a", C.c_int),
                ("precision", C.c_int), ("use_graph", C.c_int), ("stream", C.c_void_p), ("device", C.c_int),
                ("crit_sms", C.c_int), ("fp64_gemm", C.c_int)]


class PsdpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name} ({_lib().psdp_strerror(status).decode()})")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1411_3769_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        vp = C.c_void_p
        sig = {
            "psdp_default_opts": (None, [C.POINTER(Opts)]),
            "psdp_setup": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, dp, C.POINTER(Opts), C.POINTER(vp)]),
            "psdp_sizes": (C.c_int, [vp, ip]),
            "psdp_step": (C.c_int, [vp, dp]),
            "psdp_solve": (C.c_int, [vp, C.POINTER(C.c_int), dp]),
            "psdp_certify": (C.c_int, [vp, C.POINTER(C.c_int), dp, dp]),
            "psdp_grid_check": (C.c_int, [vp, C.c_int, dp, dp]),
            "psdp_get_P": (C.c_int, [vp, dp]),
            "psdp_get_y": (C.c_int, [vp, dp]),
            "psdp_get_tables": (C.c_int, [vp, ip, ip]),
            "psdp_load_iterate": (C.c_int, [vp, dp, dp, dp]),
            "psdp_get_iterate": (C.c_int, [vp, dp, dp, dp]),
            "psdp_get_schur": (C.c_int, [vp, dp]),
            "psdp_get_schur_cols": (C.c_int, [vp, ip, C.c_int, dp]),
            "psdp_apply_BT": (C.c_int, [vp, dp, dp]),
            "psdp_apply_B": (C.c_int, [vp, dp, dp]),
            "psdp_profile_enable": (C.c_int, [vp, C.c_int]),
            "psdp_profile_reset": (C.c_int, [vp]),
            "psdp_profile_get": (C.c_int, [vp, C.c_int, C.c_char_p, C.POINTER(C.c_int64), dp, C.POINTER(C.c_int)]),
            "psdp_profile_trace": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), dp, dp, C.POINTER(C.c_int),
                                             C.POINTER(C.c_int)]),
            "psdp_work": (C.c_int, [vp, dp]),
            "psdp_stream": (vp, [vp]),
            "psdp_fp64_peak": (C.c_int, [C.c_int, dp]),
            "psdp_destroy": (None, [vp]),
            "psdp_strerror": (C.c_char_p, [C.c_int]),
            "psdp_tc_gemm_check": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp]),
            "psdp_tc_gemm_persist_check": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, vp,
                                                     vp, vp]),
            "psdp_trsv_timeout_check": (C.c_int, [vp]),
            "psdp_get_schur_mixed": (C.c_int, [vp, vp]),
            "psdp_tc_gemm_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]),
            "psdp_solve_batch": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "psdp_autotune": (C.c_int, [vp, C.c_char_p, C.POINTER(C.c_int), dp]),
            "psdp_set_start": (C.c_int, [vp, dp, dp, C.c_double]),
            "psdp_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.POINTER(vp)]),
            "psdp_mlp_destroy": (None, [vp]),
            "psdp_mlp_params": (C.c_int, [vp, vp, vp, C.POINTER(C.c_int64)]),
            "psdp_mlp_grads": (C.c_int, [vp, vp, vp, C.c_int, C.POINTER(C.c_float), vp]),
            "psdp_mlp_train": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_float, C.c_uint64,
                                         C.POINTER(C.c_float)]),
            "psdp_mlp_predict": (C.c_int, [vp, vp, C.c_int, vp]),
            "psdp_fp64_peaks": (C.c_int, [C.c_int, dp, dp]),
            "psdp_engines": (C.c_int, [vp, ip]),
            "psdp_set_constant_term": (C.c_int, [vp, C.c_int, dp]),
            "psdp_set_objective": (C.c_int, [vp, dp]),
            "psdp_autotune_ex": (C.c_int, [vp, C.c_char_p, C.c_uint, C.POINTER(C.c_int), dp]),
            "psdp_ozaki_gemm_check": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_double, C.c_double,
                                                C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _check(status: int, where: str):
    if status != 0:
        raise PsdpError(status, where)


def psdp_default_opts(**kw) -> Opts:
    o = Opts()
    _lib().psdp_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def psdp_setup(n: int, l: int, d_p: int, d1: int, A: np.ndarray, opts: Opts | None = None):
    A = np.ascontiguousarray(A, dtype=np.float64)
    h = C.c_void_p()
    _check(_lib().psdp_setup(n, l, d_p, d1, _dp(A), C.byref(opts) if opts is not None else None, C.byref(h)),
           "psdp_setup")
    return h


def psdp_sizes(h) -> dict:
    out = np.zeros(9, dtype=np.int32)
    _check(_lib().psdp_sizes(h, _ip(out)), "psdp_sizes")
    return dict(zip(("n", "l", "L0", "L", "M", "Ntil", "K", "nblk", "Na"), (int(x) for x in out)))


def psdp_step(h) -> tuple[int, np.ndarray]:
    info = np.zeros(INFO_LEN)
    return _lib().psdp_step(h, _dp(info)), info


def psdp_solve(h) -> tuple[int, int, np.ndarray]:
    info = np.zeros(INFO_LEN)
    it = C.c_int(0)
    s = _lib().psdp_solve(h, C.byref(it), _dp(info))
    return s, it.value, info


def psdp_certify(h) -> tuple[int, float, float]:
    v = C.c_int(0)
    mp = np.zeros(1)
    ml = np.zeros(1)
    _check(_lib().psdp_certify(h, C.byref(v), _dp(mp), _dp(ml)), "psdp_certify")
    return v.value, float(mp[0]), float(ml[0])


def psdp_grid_check(h, N: int) -> tuple[float, float]:
    mp = np.zeros(1)
    mq = np.zeros(1)
    _check(_lib().psdp_grid_check(h, N, _dp(mp), _dp(mq)), "psdp_grid_check")
    return float(mp[0]), float(mq[0])


def psdp_get_P(h) -> np.ndarray:
    sz = psdp_sizes(h)
    P = np.zeros((sz["L0"], sz["n"], sz["n"]))
    _check(_lib().psdp_get_P(h, _dp(P)), "psdp_get_P")
    return P


def psdp_get_y(h) -> np.ndarray:
    y = np.zeros(psdp_sizes(h)["K"])
    _check(_lib().psdp_get_y(h, _dp(y)), "psdp_get_y")
    return y


def psdp_get_tables(h) -> tuple[np.ndarray, np.ndarray]:
    sz = psdp_sizes(h)
    beta = np.zeros((sz["L0"], sz["L"]), dtype=np.int32)
    c = np.zeros((sz["L0"], sz["M"], sz["Na"]), dtype=np.int32)
    _check(_lib().psdp_get_tables(h, _ip(beta), _ip(c)), "psdp_get_tables")
    return beta, c


def psdp_load_iterate(h, X: np.ndarray, Z: np.ndarray, y: np.ndarray):
    X, Z, y = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, Z, y))
    _check(_lib().psdp_load_iterate(h, _dp(X), _dp(Z), _dp(y)), "psdp_load_iterate")


def psdp_get_iterate(h):
    sz = psdp_sizes(h)
    X = np.zeros((sz["nblk"], sz["n"], sz["n"]))
    Z = np.zeros_like(X)
    y = np.zeros(sz["K"])
    _check(_lib().psdp_get_iterate(h, _dp(X), _dp(Z), _dp(y)), "psdp_get_iterate")
    return X, Z, y


def psdp_get_schur(h) -> np.ndarray:
    K = psdp_sizes(h)["K"]
    Om = np.zeros((K, K))
    _check(_lib().psdp_get_schur(h, _dp(Om)), "psdp_get_schur")
    return Om


def psdp_get_schur_cols(h, cols) -> np.ndarray:
    """Columns cols of the FP64 Schur complement at the current iterate, shape (len(cols), K)."""
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    K = psdp_sizes(h)["K"]
    out = np.zeros((len(cols), K))
    _check(_lib().psdp_get_schur_cols(h, cols.ctypes.data_as(C.POINTER(C.c_int32)), len(cols), _dp(out)),
           "psdp_get_schur_cols")
    return out


def psdp_get_schur_mixed(h) -> np.ndarray:
    K = psdp_sizes(h)["K"]
    Om = np.zeros((K, K), dtype=np.float32)
    _check(_lib().psdp_get_schur_mixed(h, Om.ctypes.data), "psdp_get_schur_mixed")
    return Om


def psdp_apply_BT(h, v: np.ndarray) -> np.ndarray:
    sz = psdp_sizes(h)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros((sz["nblk"], sz["n"], sz["n"]))
    _check(_lib().psdp_apply_BT(h, _dp(v), _dp(out)), "psdp_apply_BT")
    return out


def psdp_apply_B(h, W: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros(psdp_sizes(h)["K"])
    _check(_lib().psdp_apply_B(h, _dp(W), _dp(out)), "psdp_apply_B")
    return out


def psdp_profile_enable(h, on: bool = True):
    _check(_lib().psdp_profile_enable(h, int(on)), "psdp_profile_enable")


def psdp_profile_reset(h):
    _check(_lib().psdp_profile_reset(h), "psdp_profile_reset")


def psdp_profile_get(h, max_entries: int = 64) -> dict:
    names = C.create_string_buffer(32 * max_entries)
    launches = np.zeros(max_entries, dtype=np.int64)
    ms = np.zeros(max_entries)
    cnt = C.c_int(0)
    _check(_lib().psdp_profile_get(h, max_entries, names, launches.ctypes.data_as(C.POINTER(C.c_int64)), _dp(ms),
                                   C.byref(cnt)), "psdp_profile_get")
    out = {}
    raw = names.raw
    for i in range(cnt.value):
        nm = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def psdp_profile_trace(h, max_entries: int = 20000) -> list:
    """[(name, t0_ms, t1_ms, on_crit)] of the last profiled step, in issue order."""
    names = list(psdp_profile_get(h, 256).keys())
    ids = np.zeros(max_entries, dtype=np.int32)
    t0 = np.zeros(max_entries)
    t1 = np.zeros(max_entries)
    crit = np.zeros(max_entries, dtype=np.int32)
    cnt = C.c_int(0)
    ip = C.POINTER(C.c_int)
    _check(_lib().psdp_profile_trace(h, max_entries, ids.ctypes.data_as(ip), _dp(t0), _dp(t1), crit.ctypes.data_as(ip),
                                     C.byref(cnt)), "psdp_profile_trace")
    return [(names[ids[i]], float(t0[i]), float(t1[i]), bool(crit[i])) for i in range(cnt.value)]


def psdp_work(h) -> dict:
    out = np.zeros(7)
    _check(_lib().psdp_work(h, _dp(out)), "psdp_work")
    return dict(schur_flops=out[0], chol_flops=out[1], schur_terms=out[2], schur_dense_flops=out[3],
                kernels_per_step=int(out[4]), nb_chol=int(out[5]), nb_chol32=int(out[6]))


def psdp_set_constant_term(h, d_r: int, R: np.ndarray) -> None:
    R = np.ascontiguousarray(R, dtype=np.float64)
    _check(_lib().psdp_set_constant_term(h, d_r, _dp(R)), "psdp_set_constant_term")


def psdp_set_objective(h, a: np.ndarray) -> None:
    a = np.ascontiguousarray(a, dtype=np.float64)
    _check(_lib().psdp_set_objective(h, _dp(a)), "psdp_set_objective")


def psdp_engines(h) -> dict:
    out = np.zeros(2, dtype=np.int32)
    _check(_lib().psdp_engines(h, _ip(out)), "psdp_engines")
    return dict(schur="ozaki" if out[0] else "dfma", cholesky="ozaki" if out[1] else "dfma")


def psdp_stream(h) -> int:
    return _lib().psdp_stream(h) or 0


def psdp_fp64_peak(device: int = 0) -> float:
    v = np.zeros(1)
    _check(_lib().psdp_fp64_peak(device, _dp(v)), "psdp_fp64_peak")
    return float(v[0])


def psdp_fp64_peaks(device: int = 0) -> tuple[float, float]:
    """(DFMA, DMMA) FP64 TFLOP/s of this GPU."""
    a, b = np.zeros(1), np.zeros(1)
    _check(_lib().psdp_fp64_peaks(device, _dp(a), _dp(b)), "psdp_fp64_peaks")
    return float(a[0]), float(b[0])


def psdp_ozaki_gemm_check(A: np.ndarray, B: np.ndarray, C0: np.ndarray | None = None, alpha: float = 1.0,
                          beta: float = 0.0, lower: bool = False) -> np.ndarray:
    """alpha A B^T + beta C0 (M x N, FP64) through the Ozaki-scheme tensor-core product."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    Ct = np.ascontiguousarray((np.zeros((M, N)) if C0 is None else np.asarray(C0, dtype=np.float64)).T)
    _check(_lib().psdp_ozaki_gemm_check(M, N, K, _dp(A), _dp(B), _dp(Ct), alpha, beta, int(lower)),
           "psdp_ozaki_gemm_check")
    return Ct.T


def psdp_tc_gemm_check(A: np.ndarray, B: np.ndarray, split: int = 1) -> np.ndarray:
    """D = A B^T on the tensor cores; A, B float32 (TF32 / 3xTF32) or uint16 BF16 bit patterns."""
    dtype = 1 if A.dtype == np.uint16 else 0
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    M, K = A.shape
    N = B.shape[0]
    C_ = np.zeros((N, M), dtype=np.float32)
    _check(_lib().psdp_tc_gemm_check(M, N, K, dtype, split, A.ctypes.data, B.ctypes.data, C_.ctypes.data),
           "psdp_tc_gemm_check")
    return C_.T


def psdp_tc_gemm_persist_check(A: np.ndarray, B: np.ndarray, C0: np.ndarray, split: int = 3, tri: int = 1,
                               ctas: int = 152, timing: bool = False):
    """C0 - A B^T on the (lower-triangular when tri) 128 x 128 tiles by the persistent kernel; float32.
    With timing=True also returns the kernel's duration in ms."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    M, K = A.shape
    N = B.shape[0]
    C_ = np.ascontiguousarray(np.asarray(C0, dtype=np.float32).T)    # [N][M]: C[n*M + m]
    ms = np.zeros(1, dtype=np.float32)
    _check(_lib().psdp_tc_gemm_persist_check(M, N, K, split, tri, ctas, A.ctypes.data, B.ctypes.data,
                                             C_.ctypes.data, ms.ctypes.data), "psdp_tc_gemm_persist_check")
    return (C_.T, float(ms[0])) if timing else C_.T


def psdp_trsv_timeout_check() -> tuple[str, float]:
    """Status name and the kernel's duration in ms of the bounded-wait self-test."""
    ms = np.zeros(1, dtype=np.float32)
    s = _lib().psdp_trsv_timeout_check(ms.ctypes.data)
    return STATUS.get(s, str(s)), float(ms[0])


def psdp_tc_gemm_noalloc(M: int, N: int, K: int, split: int, A_ptr: int, B_ptr: int, C_ptr: int,
                         stream: int = 0) -> int:
    """Device pointers in and out; returns the status code (no allocation inside)."""
    return _lib().psdp_tc_gemm_noalloc(M, N, K, split, A_ptr, B_ptr, C_ptr, stream or None)


def psdp_solve_batch(handles) -> tuple[list[str], list[int]]:
    n = len(handles)
    arr = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    st = (C.c_int * n)()
    it = (C.c_int * n)()
    _check(_lib().psdp_solve_batch(arr, n, st, it), "psdp_solve_batch")
    return [STATUS[s] for s in st], list(it)


def psdp_autotune(h, cache_path: str | None = None) -> tuple[int, np.ndarray]:
    ch = C.c_int(-1)
    ms = np.zeros(3)
    _check(_lib().psdp_autotune(h, cache_path.encode() if cache_path else None, C.byref(ch), _dp(ms)),
           "psdp_autotune")
    return ch.value, ms


TUNE_CANDIDATES = ("fp64-auto", "mixed-64", "mixed-128", "fp64-fma", "fp64-ozaki", "fp64-ozaki-schur")


def psdp_autotune_ex(h, mask: int, cache_path: str | None = None) -> tuple[int, np.ndarray]:
    ch = C.c_int(-1)
    ms = np.zeros(len(TUNE_CANDIDATES))
    _check(_lib().psdp_autotune_ex(h, cache_path.encode() if cache_path else None, mask, C.byref(ch), _dp(ms)),
           "psdp_autotune_ex")
    return ch.value, ms


def psdp_set_start(h, y0: np.ndarray, xscale: np.ndarray | None, theta: float):
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    xs = None if xscale is None else np.ascontiguousarray(xscale, dtype=np.float64)
    _check(_lib().psdp_set_start(h, _dp(y0), _dp(xs) if xs is not None else None, theta), "psdp_set_start")


def _fp(a: np.ndarray) -> int:
    return a.ctypes.data


def psdp_mlp_create(n_in: int, width: int, n_out: int, max_batch: int, seed: int = 0, device: int = 0):
    h = C.c_void_p()
    _check(_lib().psdp_mlp_create(n_in, width, n_out, max_batch, seed, device, C.byref(h)), "psdp_mlp_create")
    return h


def psdp_mlp_destroy(h):
    if h:
        _lib().psdp_mlp_destroy(h)


def psdp_mlp_params(h, set_to: np.ndarray | None = None) -> np.ndarray:
    cnt = C.c_int64(0)
    _check(_lib().psdp_mlp_params(h, None, None, C.byref(cnt)), "psdp_mlp_params")
    out = np.zeros(cnt.value, dtype=np.float32)
    src = None if set_to is None else np.ascontiguousarray(set_to, dtype=np.float32)
    _check(_lib().psdp_mlp_params(h, _fp(out), _fp(src) if src is not None else None, None), "psdp_mlp_params")
    return out


def psdp_mlp_grads(h, X: np.ndarray, T: np.ndarray) -> tuple[float, np.ndarray]:
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    cnt = C.c_int64(0)
    _check(_lib().psdp_mlp_params(h, None, None, C.byref(cnt)), "psdp_mlp_params")
    g = np.zeros(cnt.value, dtype=np.float32)
    loss = C.c_float(0.0)
    _check(_lib().psdp_mlp_grads(h, _fp(X), _fp(T), X.shape[0], C.byref(loss), _fp(g)), "psdp_mlp_grads")
    return float(loss.value), g


def psdp_mlp_train(h, X: np.ndarray, T: np.ndarray, epochs: int, batch: int, lr: float, seed: int = 0) -> float:
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    loss = C.c_float(0.0)
    _check(_lib().psdp_mlp_train(h, _fp(X), _fp(T), X.shape[0], epochs, batch, lr, seed, C.byref(loss)),
           "psdp_mlp_train")
    return float(loss.value)


def psdp_mlp_predict(h, X: np.ndarray, n_out: int) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.zeros((X.shape[0], n_out), dtype=np.float32)
    _check(_lib().psdp_mlp_predict(h, _fp(X), X.shape[0], _fp(Y)), "psdp_mlp_predict")
    return Y


def psdp_destroy(h):
    if h:
        _lib().psdp_destroy(h)


def psdp_strerror(status: int) -> str:
    return _lib().psdp_strerror(status).decode()


class Solver:
    """Owning handle: ``Solver(A, d_p, d1, **opts)`` then ``.solve()``, ``.certify()``."""

    def __init__(self, A: np.ndarray, d_p: int, d1: int, **opts):
        A = np.asarray(A, dtype=np.float64)
        self.n = A.shape[-1]
        d_a = opts.get("d_a", 1)
        self.l = opts.pop("l", None) or _infer_l(A.shape[0], d_a)
        self.h = psdp_setup(self.n, self.l, d_p, d1, A, psdp_default_opts(**opts))
        self.sizes = psdp_sizes(self.h)

    def step(self) -> dict:
        s, info = psdp_step(self.h)
        _check(s, "psdp_step")
        return dict(zip(INFO_FIELDS, info))

    def solve(self) -> tuple[str, int, dict]:
        s, it, info = psdp_solve(self.h)
        if s not in (0, 6, 8):
            raise PsdpError(s, "psdp_solve")
        return STATUS[s], it, dict(zip(INFO_FIELDS, info))

    def certify(self):
        return psdp_certify(self.h)

    def close(self):
        psdp_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.close()
        except Exception:
            pass


def _infer_l(Na: int, d_a: int) -> int:
    from math import comb
    l = 1
    while comb(l + d_a - 1, l - 1) < Na:
        l += 1
    return l
