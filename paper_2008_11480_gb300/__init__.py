"""GB300-native factorized high-order Newton-Schulz inversion coupled to
Richardson iteration (A. Stotsky, arXiv 2008.11480).

This module is a thin ctypes binding over ``libnsgb.so`` (C ABI declared in
``include/nsgb.h``): it marshals torch tensors (device or host) into pointers
and sizes and calls the library; every step of the method runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
the calls raise.

Functions keep the ABI names (``ns_create``, ``ns_invert``,
``ns_richardson_solve``, ``ns_residual``, and the single-kernel ``ns_k_*``).
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import torch

__all__ = [
    "NS_OK", "NS_NOT_CONVERGED", "NS_ERR_ARG", "NS_ERR_CUDA", "NS_ERR_OOM", "NS_ERR_DIVERGED",
    "NS_ERR_TIMEOUT", "NS_ERR_NONFINITE", "NS_ERR_UNSUPPORTED",
    "NS_FP64", "NS_BF16", "NS_BF16X3", "NS_AUTO",
    "NSError", "ns_options", "ns_stats", "lib", "lib_path", "header_path", "default_options",
    "ns_create", "ns_destroy", "ns_set_stream", "ns_invert", "ns_richardson_solve", "ns_residual",
    "ns_inverse_residual",
    "ns_last_error", "ns_status_string", "ns_k_split", "ns_k_gemm_bf16", "ns_k_gemm_f64", "ns_k_resid",
    "ns_k_split3", "ns_k_gemm_bf16x6", "NS_BF16X6", "NS_BF16X2", "ns_k_gemm_oz", "ns_k_gemm_tf32", "NS_TF32",
    "ns_k_update", "ns_k_prep_a", "ns_k_resid_x2", "ns_k_resid_noalloc", "Context",
    "ns_batch_stats", "Batch",
]

NS_OK, NS_NOT_CONVERGED = 0, 1
NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_OOM, NS_ERR_DIVERGED = -1, -2, -3, -4
NS_ERR_TIMEOUT, NS_ERR_NONFINITE, NS_ERR_UNSUPPORTED = -5, -6, -7
NS_FP64, NS_TF32, NS_BF16, NS_BF16X3, NS_BF16X6, NS_AUTO, NS_BF16X2 = 0, 1, 2, 3, 4, 5, 6
NS_MAX_HIST = 256

_PKG = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_PKG, "libnsgb.so")
header_path = os.path.join(os.path.dirname(_PKG), "include", "nsgb.h")


class NSError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{_status_name(status)}: {msg}" if msg else _status_name(status))


class ns_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("form", ctypes.c_int),
        ("pow_mode", ctypes.c_int),
        ("g0_mode", ctypes.c_int),
        ("ns_stop", ctypes.c_int),
        ("ns_stop_frob", ctypes.c_double),
        ("max_sweeps", ctypes.c_int),
        ("use_updated_G", ctypes.c_int),
        ("profile", ctypes.c_int),
        ("gemm_bn", ctypes.c_int),
        ("timeout_s", ctypes.c_double),
        ("aux_ahead", ctypes.c_int),
        ("gemm_cluster", ctypes.c_int),
        ("couple_frob", ctypes.c_double),
        ("accel_richardson", ctypes.c_int),
        ("g0_order", ctypes.c_int),
        ("final_check", ctypes.c_int),
        ("fp64_slices", ctypes.c_int),
        ("fp64_slices_early", ctypes.c_int),
        ("pow_bf16", ctypes.c_int),
        ("tf32_rung", ctypes.c_int),
        ("fp64_slices_pow", ctypes.c_int),
        ("batch_fused", ctypes.c_int),
        ("xp_bf16x2", ctypes.c_int),
    ]


class ns_stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("ns_iters", ctypes.c_int),
        ("sweeps", ctypes.c_int),
        ("rollbacks", ctypes.c_int),
        ("n_frob", ctypes.c_int),
        ("n_res", ctypes.c_int),
        ("rel_res", ctypes.c_double),
        ("frob_F", ctypes.c_double * NS_MAX_HIST),
        ("prec_hist", ctypes.c_int * NS_MAX_HIST),
        ("rel_res_hist", ctypes.c_double * NS_MAX_HIST),
        ("gemm_launches", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("gemm_flops", ctypes.c_double),
        ("gemm_ms", ctypes.c_double),
        ("tc_gemm_ms", ctypes.c_double),
        ("tc_gemm_launches", ctypes.c_longlong),
        ("tc_gemm_flops", ctypes.c_double),
        ("wall_ms", ctypes.c_double),
        ("final_frob", ctypes.c_double),
        ("tc_gemm_alg_flops", ctypes.c_double),
        ("slice_pair_flops", ctypes.c_double),
    ]

    def frob_history(self) -> list[float]:
        return [self.frob_F[i] for i in range(self.n_frob)]

    def prec_history(self) -> list[int]:
        return [self.prec_hist[i] for i in range(self.n_frob)]

    def res_history(self) -> list[float]:
        return [self.rel_res_hist[i] for i in range(self.n_res)]


class ns_batch_stats(ctypes.Structure):
    _fields_ = [
        ("passes", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("not_converged", ctypes.c_int),
        ("gemm_launches", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("gemm_flops", ctypes.c_double),
        ("gemm_ms", ctypes.c_double),
        ("useful_flops_per_product", ctypes.c_double),
        ("wall_ms", ctypes.c_double),
        ("gemm_bytes", ctypes.c_double),
        ("fused", ctypes.c_int),
        ("fused_pad", ctypes.c_int),
        ("fused_ms", ctypes.c_double),
        ("useful_flops", ctypes.c_double),
        ("slice_retried", ctypes.c_int),
        ("slice_retried_converged", ctypes.c_int),
        ("slice_retry_ms", ctypes.c_double),
    ]


class ns_request(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nrhs", ctypes.c_int),
        ("iters", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("A", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("Theta", ctypes.c_void_p),
    ]


class ns_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("done", ctypes.c_int),
        ("ns_iters", ctypes.c_int),
        ("sweeps", ctypes.c_int),
        ("rel_res", ctypes.c_double),
        ("queue_ms", ctypes.c_double),
        ("latency_ms", ctypes.c_double),
    ]


class ns_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong),
        ("admitted", ctypes.c_longlong),
        ("completed", ctypes.c_longlong),
        ("converged", ctypes.c_longlong),
        ("rejected", ctypes.c_longlong),
        ("ticks", ctypes.c_longlong),
        ("passes", ctypes.c_longlong),
        ("active", ctypes.c_int),
        ("queued", ctypes.c_int),
        ("last_error", ctypes.c_int),
        ("gemm_launches", ctypes.c_longlong),
        ("kernel_launches", ctypes.c_longlong),
        ("gemm_flops", ctypes.c_double),
        ("tick_ms", ctypes.c_double),
        ("wait_ms", ctypes.c_double),
    ]


_LIB = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


def lib() -> ctypes.CDLL:
    """Load libnsgb.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(lib_path):
        raise RuntimeError(f"{lib_path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(lib_path)
    sig = {
        "ns_default_options": (None, [ctypes.POINTER(ns_options)]),
        "ns_create": (_int, [_i64, _int, ctypes.POINTER(_int), _int, ctypes.POINTER(ns_options), ctypes.POINTER(_vp)]),
        "ns_destroy": (_int, [_vp]),
        "ns_set_stream": (_int, [_vp, _vp]),
        "ns_invert": (_int, [_vp, _vp, _vp, _int, _vp, ctypes.POINTER(ns_stats)]),
        "ns_richardson_solve": (_int, [_vp, _vp, _vp, _int, _vp, _int, ctypes.c_double, _vp, ctypes.POINTER(ns_stats)]),
        "ns_residual": (_int, [_vp, _vp, _vp, _vp, _int, _vp]),
        "ns_inverse_residual": (_int, [_vp, _vp, _vp, _int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
        "ns_last_error": (ctypes.c_char_p, [_vp]),
        "ns_status_string": (ctypes.c_char_p, [_int]),
        "ns_k_split": (_int, [_vp, _int, _i64, _i64, _i64, _vp, _vp, _i64, _vp]),
        "ns_k_split3": (_int, [_vp, _int, _i64, _i64, _i64, _vp, _vp, _vp, _i64, _vp]),
        "ns_k_gemm_oz": (_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, ctypes.c_double, _vp, _i64, ctypes.c_double,
                                 ctypes.c_double, _vp, _i64, _int, _vp, _vp]),
        "ns_k_gemm_tf32": (_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, ctypes.c_float, _vp, _i64, ctypes.c_float,
                                   ctypes.c_float, _vp, _i64, _vp, _vp, _i64, _vp, _vp]),
        "ns_k_gemm_bf16x6": (_int, [_i64, _i64, _i64, ctypes.POINTER(_vp), _i64, ctypes.POINTER(_vp), _i64,
                                     ctypes.c_float, _vp, _i64, ctypes.c_float, ctypes.c_float, _vp, _i64,
                                     ctypes.POINTER(_vp), _i64, _vp, _vp]),
        "ns_k_gemm_bf16": (_int, [_int, _i64, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _i64, ctypes.c_float, _vp, _i64,
                                  ctypes.c_float, ctypes.c_float, _vp, _i64, _vp, _vp, _i64, _vp, _int, _int, _vp]),
        "ns_k_gemm_f64": (_int, [_i64, _i64, _i64, _vp, _i64, _vp, _i64, ctypes.c_double, _vp, _i64, ctypes.c_double,
                                 ctypes.c_double, _vp, _i64, _vp, _vp]),
        "ns_k_resid": (_int, [_vp, _i64, _vp, _vp, _vp, _i64, _int, _vp, _vp]),
        "ns_k_update": (_int, [_vp, _int, _i64, _vp, _vp, _i64, _int, _vp]),
        "ns_k_prep_a": (_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
        "ns_k_resid_x2": (_int, [_vp, _vp, _i64, _vp, _vp, _vp, _i64, _int, _vp, _vp]),
        "ns_k_resid_noalloc": (_int, [_vp, _i64, _vp, _vp, _vp, _i64, _int, _vp, _vp]),
        "ns_batch_create": (_int, [_int, ctypes.POINTER(_i64), ctypes.POINTER(_int), _int, ctypes.POINTER(ns_options),
                                   ctypes.POINTER(_vp)]),
        "ns_batch_destroy": (_int, [_vp]),
        "ns_batch_set_stream": (_int, [_vp, _vp]),
        "ns_batch_last_error": (ctypes.c_char_p, [_vp]),
        "ns_batch_solve": (_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _int,
                                  ctypes.c_double, ctypes.POINTER(ns_batch_stats)]),
        "ns_batch_result": (_int, [_vp, _int, ctypes.POINTER(_int), ctypes.POINTER(_int), ctypes.POINTER(_int),
                                   ctypes.POINTER(ctypes.c_double)]),
        "ns_server_create": (_int, [ctypes.c_size_t, _int, _int, _int, ctypes.POINTER(ns_options),
                                    ctypes.POINTER(_vp)]),
        "ns_server_destroy": (_int, [_vp]),
        "ns_server_set_stream": (_int, [_vp, _vp]),
        "ns_server_last_error": (ctypes.c_char_p, [_vp]),
        "ns_server_submit": (_int, [_vp, ctypes.POINTER(ns_request), ctypes.POINTER(ctypes.c_uint64)]),
        "ns_server_poll": (_int, [_vp, ctypes.c_uint64, ctypes.POINTER(ns_result)]),
        "ns_server_release": (_int, [_vp, ctypes.c_uint64]),
        "ns_server_tick": (_int, [_vp, ctypes.POINTER(_int)]),
        "ns_server_start": (_int, [_vp]),
        "ns_server_stop": (_int, [_vp]),
        "ns_server_get_stats": (_int, [_vp, ctypes.POINTER(ns_server_stats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def declared_functions() -> list[str]:
    """Names of the functions include/nsgb.h declares."""
    txt = open(header_path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ns_[a-z0-9_]+)\s*\(", txt, re.M)))


def _status_name(s: int) -> str:
    try:
        return lib().ns_status_string(s).decode()
    except Exception:
        return f"status {s}"


def ns_status_string(s: int) -> str:
    return lib().ns_status_string(s).decode()


def default_options(**kw) -> ns_options:
    o = ns_options()
    lib().ns_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _ptr(t: torch.Tensor | None, dtype=torch.float64) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def ns_create(n: int, order: int, rates=(), opt: ns_options | None = None) -> int:
    arr = (_int * max(1, len(rates)))(*rates) if rates else None
    h = _vp()
    s = lib().ns_create(int(n), int(order), arr, len(rates), ctypes.byref(opt) if opt is not None else None,
                        ctypes.byref(h))
    if s != NS_OK:
        raise NSError(s, "ns_create")
    return h.value


def ns_destroy(ctx: int) -> None:
    lib().ns_destroy(ctx)


def ns_set_stream(ctx: int, stream) -> None:
    s = lib().ns_set_stream(ctx, _stream_ptr(stream))
    if s != NS_OK:
        raise NSError(s)


def ns_last_error(ctx: int) -> str:
    return lib().ns_last_error(ctx).decode()


def _check(ctx: int, s: int, allow=(NS_OK, NS_NOT_CONVERGED)) -> int:
    if s not in allow:
        raise NSError(s, ns_last_error(ctx))
    return s


def ns_invert(ctx: int, A: torch.Tensor, G0: torch.Tensor | None, iters: int, G_out: torch.Tensor | None,
              check: bool = True) -> tuple[int, ns_stats]:
    st = ns_stats()
    s = lib().ns_invert(ctx, _ptr(A), _ptr(G0), int(iters), _ptr(G_out), ctypes.byref(st))
    if check:
        _check(ctx, s)
    return s, st


def ns_richardson_solve(ctx: int, A: torch.Tensor, B: torch.Tensor, theta0: torch.Tensor | None, iters: int,
                        tol: float, theta_out: torch.Tensor, check: bool = True) -> tuple[int, ns_stats]:
    st = ns_stats()
    nrhs = B.shape[1] if B.dim() == 2 else 1
    s = lib().ns_richardson_solve(ctx, _ptr(A), _ptr(B), nrhs, _ptr(theta0), int(iters), float(tol),
                                  _ptr(theta_out), ctypes.byref(st))
    if check:
        _check(ctx, s)
    return s, st


def ns_residual(ctx: int, A: torch.Tensor, theta: torch.Tensor, B: torch.Tensor) -> list[float]:
    nrhs = B.shape[1] if B.dim() == 2 else 1
    out = (ctypes.c_double * nrhs)()
    s = lib().ns_residual(ctx, _ptr(A), _ptr(theta), _ptr(B), nrhs, out)
    _check(ctx, s, (NS_OK,))
    return list(out)


def ns_inverse_residual(ctx: int, A: torch.Tensor, G: torch.Tensor, probes: int = 0, seed: int = 0) -> float:
    """||I - A G||_F in FP64: exact (probes = 0) or Hutchinson's estimate with
    `probes` Rademacher probes drawn from SplitMix64 at `seed`."""
    out = ctypes.c_double(0.0)
    s = lib().ns_inverse_residual(ctx, _ptr(A), _ptr(G), int(probes), int(seed) & (2 ** 64 - 1), ctypes.byref(out))
    _check(ctx, s, (NS_OK,))
    return out.value


# ---------------------------------------------------------------- single kernels

def _raise(s: int, what: str):
    if s != NS_OK:
        raise NSError(s, what)


def ns_k_split(X: torch.Tensor, hi: torch.Tensor, lo: torch.Tensor, rows: int, cols: int, ldx: int, ld: int,
               stream=None) -> None:
    dt = {torch.float64: 0, torch.float32: 1}[X.dtype]
    _raise(lib().ns_k_split(X.data_ptr(), dt, rows, cols, ldx, _ptr(hi, torch.bfloat16), _ptr(lo, torch.bfloat16),
                            ld, _stream_ptr(stream)), "ns_k_split")


def ns_k_split3(X: torch.Tensor, hi: torch.Tensor, lo: torch.Tensor, lo2: torch.Tensor, rows: int, cols: int,
                ldx: int, ld: int, stream=None) -> None:
    dt = {torch.float64: 0, torch.float32: 1}[X.dtype]
    bf = torch.bfloat16
    _raise(lib().ns_k_split3(X.data_ptr(), dt, rows, cols, ldx, _ptr(hi, bf), _ptr(lo, bf), _ptr(lo2, bf), ld,
                             _stream_ptr(stream)), "ns_k_split3")


def ns_k_gemm_bf16x6(M: int, N: int, K: int, L, ldl: int, R, ldr: int, s: float = 1.0, C=None, ldc: int = 0,
                     beta: float = 0.0, gamma: float = 0.0, D32=None, ldd32: int = 0, D=None, ldd16: int = 0,
                     frob_out=None, stream=None) -> None:
    """L, R: sequences of the three bf16 parts (hi, lo, lo2); D: None or three
    optional bf16 outputs."""
    bf = torch.bfloat16
    Lp = (_vp * 3)(*[_ptr(x, bf) for x in L])
    Rp = (_vp * 3)(*[_ptr(x, bf) for x in R])
    Dp = None if D is None else (_vp * 3)(*[_ptr(x, bf) for x in D])
    r = lib().ns_k_gemm_bf16x6(M, N, K, Lp, ldl, Rp, ldr, s, _ptr(C, torch.float32), ldc, beta, gamma,
                               _ptr(D32, torch.float32), ldd32, Dp, ldd16, _ptr(frob_out), _stream_ptr(stream))
    _raise(r, "ns_k_gemm_bf16x6")


def ns_k_gemm_tf32(M: int, N: int, K: int, L, ldl: int, R, ldr: int, s: float = 1.0, C=None, ldc: int = 0,
                   beta: float = 0.0, gamma: float = 0.0, D32=None, ldd32: int = 0, Dt=None, DtT=None, ldt: int = 0,
                   frob_out=None, stream=None) -> None:
    """TF32 tensor-core product with the Newton-Schulz epilogue (f32 tensors)."""
    f = torch.float32
    r = lib().ns_k_gemm_tf32(M, N, K, _ptr(L, f), ldl, _ptr(R, f), ldr, s, _ptr(C, f), ldc, beta, gamma,
                             _ptr(D32, f), ldd32, _ptr(Dt, f), _ptr(DtT, f), ldt, _ptr(frob_out), _stream_ptr(stream))
    _raise(r, "ns_k_gemm_tf32: " + lib().ns_last_error(None).decode())


def ns_k_gemm_oz(M: int, N: int, K: int, L, ldl: int, R, ldr: int, s: float = 1.0, C=None, ldc: int = 0,
                 beta: float = 0.0, gamma: float = 0.0, D=None, ldd: int = 0, slices: int = 7, frob_out=None,
                 stream=None) -> None:
    """FP64-accurate product from integer bf16 slices on the tensor cores (FP64 tensors)."""
    r = lib().ns_k_gemm_oz(M, N, K, _ptr(L), ldl, _ptr(R), ldr, s, _ptr(C), ldc, beta, gamma, _ptr(D), ldd, slices,
                           _ptr(frob_out), _stream_ptr(stream))
    _raise(r, "ns_k_gemm_oz: " + lib().ns_last_error(None).decode())


def ns_k_gemm_bf16(precision: int, M: int, N: int, K: int, Lhi, Llo, ldl: int, Rhi, Rlo, ldr: int, s: float = 1.0,
                   C=None, ldc: int = 0, beta: float = 0.0, gamma: float = 0.0, D32=None, ldd32: int = 0,
                   Dhi=None, Dlo=None, ldd16: int = 0, frob_out=None, bn: int = 0, cluster_m: int = 0,
                   stream=None) -> None:
    bf = torch.bfloat16
    r = lib().ns_k_gemm_bf16(precision, M, N, K, _ptr(Lhi, bf), _ptr(Llo, bf), ldl, _ptr(Rhi, bf), _ptr(Rlo, bf), ldr,
                             s, _ptr(C, torch.float32), ldc, beta, gamma, _ptr(D32, torch.float32), ldd32,
                             _ptr(Dhi, bf), _ptr(Dlo, bf), ldd16, _ptr(frob_out), bn, cluster_m, _stream_ptr(stream))
    _raise(r, "ns_k_gemm_bf16")


def ns_k_gemm_f64(M: int, N: int, K: int, L, ldl: int, R, ldr: int, s: float, C, ldc: int, beta: float, gamma: float,
                  D, ldd: int, frob_out=None, stream=None) -> None:
    r = lib().ns_k_gemm_f64(M, N, K, _ptr(L), ldl, _ptr(R), ldr, s, _ptr(C), ldc, beta, gamma, _ptr(D), ldd,
                            _ptr(frob_out), _stream_ptr(stream))
    _raise(r, "ns_k_gemm_f64")


def ns_k_resid(A, lda: int, theta, B, R, n: int, nrhs: int, rsq_out=None, stream=None) -> None:
    _raise(lib().ns_k_resid(_ptr(A), lda, _ptr(theta), _ptr(B), _ptr(R), n, nrhs, _ptr(rsq_out),
                            _stream_ptr(stream)), "ns_k_resid")


def ns_k_resid_noalloc(A, lda: int, theta, B, R, n: int, nrhs: int, rsq_out=None, stream=None) -> int:
    """ns_k_resid without any device allocation (fixed scratch; n <= 32768,
    nrhs <= 16).  Returns the status instead of raising on NS_ERR_ARG."""
    s = lib().ns_k_resid_noalloc(_ptr(A), lda, _ptr(theta), _ptr(B), _ptr(R), n, nrhs, _ptr(rsq_out),
                                 _stream_ptr(stream))
    if s not in (NS_OK, NS_ERR_ARG):
        raise NSError(s, "ns_k_resid_noalloc")
    return s


def ns_k_update(G, ldg: int, R, theta, n: int, nrhs: int, stream=None) -> None:
    dt = {torch.float64: 0, torch.float32: 1}[G.dtype]
    _raise(lib().ns_k_update(G.data_ptr(), dt, ldg, _ptr(R), _ptr(theta), n, nrhs, _stream_ptr(stream)),
           "ns_k_update")


def ns_k_prep_a(A, lda: int, n: int, hi, lo, a1, a2, ld: int, ss_out=None, rowabs_out=None, stream=None) -> None:
    bf = torch.bfloat16
    _raise(lib().ns_k_prep_a(_ptr(A), lda, n, _ptr(hi, bf), _ptr(lo, bf), _ptr(a1, torch.float32),
                             _ptr(a2, torch.float32), ld, _ptr(ss_out), _ptr(rowabs_out), _stream_ptr(stream)),
           "ns_k_prep_a")


def ns_k_resid_x2(a1, a2, ld: int, theta, B, R, n: int, nrhs: int, rsq_out=None, stream=None) -> None:
    _raise(lib().ns_k_resid_x2(_ptr(a1, torch.float32), _ptr(a2, torch.float32), ld, _ptr(theta), _ptr(B), _ptr(R),
                               n, nrhs, _ptr(rsq_out), _stream_ptr(stream)), "ns_k_resid_x2")


# ---------------------------------------------------------------- convenience

@dataclass
class SolveResult:
    theta: torch.Tensor
    status: int
    stats: ns_stats


class Context:
    """Owns one ``ns_ctx``: ``Context(n, order=4, rates=(), **options)``."""

    def __init__(self, n: int, order: int = 4, rates=(), stream=None, **options):
        self.n = int(n)
        self.opt = default_options(**options)
        self.handle = ns_create(n, order, tuple(rates), self.opt)
        if stream is not None:
            ns_set_stream(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            ns_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def invert(self, A: torch.Tensor, iters: int, G0: torch.Tensor | None = None,
               out: torch.Tensor | None = None) -> tuple[torch.Tensor, ns_stats]:
        if out is None:
            out = torch.empty((self.n, self.n), dtype=torch.float64, device=A.device)
        _, st = ns_invert(self.handle, A, G0, iters, out)
        return out, st

    def solve(self, A: torch.Tensor, B: torch.Tensor, iters: int = 64, tol: float = 1e-10,
              theta0: torch.Tensor | None = None, out: torch.Tensor | None = None) -> SolveResult:
        if out is None:
            out = torch.empty_like(B)
        s, st = ns_richardson_solve(self.handle, A, B, theta0, iters, tol, out)
        return SolveResult(out, s, st)

    def residual(self, A, theta, B) -> list[float]:
        return ns_residual(self.handle, A, theta, B)

    def inverse_residual(self, A, G, probes: int = 0, seed: int = 0) -> float:
        return ns_inverse_residual(self.handle, A, G, probes, seed)


class Batch:
    """Many independent SPD systems solved together (``ns_batch_*``).

    ``Batch(ns, nrhs, order=4, **options)`` allocates the workspace; ``solve``
    takes lists of device FP64 tensors A_i (n_i x n_i), B_i (n_i x nrhs_i) and
    returns the Theta_i (device tensors) with the per-instance outcomes."""

    def __init__(self, ns, nrhs, order: int = 4, stream=None, **options):
        self.count = len(ns)
        self.ns = [int(x) for x in ns]
        self.nrhs = [int(x) for x in nrhs]
        self.opt = default_options(**options)
        h = _vp()
        n_arr = (_i64 * self.count)(*self.ns)
        r_arr = (_int * self.count)(*self.nrhs)
        s = lib().ns_batch_create(self.count, n_arr, r_arr, int(order), ctypes.byref(self.opt), ctypes.byref(h))
        if s != NS_OK:
            raise NSError(s, "ns_batch_create")
        self.handle = h.value
        if stream is not None:
            lib().ns_batch_set_stream(self.handle, _stream_ptr(stream))

    def close(self):
        if getattr(self, "handle", None):
            lib().ns_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, As, Bs, iters: int = 64, tol: float = 1e-10, outs=None):
        if outs is None:
            outs = [torch.empty_like(Bi) for Bi in Bs]
        for i, (Ai, Bi, Ti) in enumerate(zip(As, Bs, outs)):
            if not (Ai.is_cuda and Bi.is_cuda and Ti.is_cuda):
                raise ValueError("batched solves take device tensors")
            _ptr(Ai), _ptr(Bi), _ptr(Ti)
            if Ai.shape != (self.ns[i], self.ns[i]) or Bi.shape != (self.ns[i], self.nrhs[i]):
                raise ValueError(f"instance {i}: shape mismatch")
        a = (_vp * self.count)(*[t.data_ptr() for t in As])
        b = (_vp * self.count)(*[t.data_ptr() for t in Bs])
        o = (_vp * self.count)(*[t.data_ptr() for t in outs])
        st = ns_batch_stats()
        s = lib().ns_batch_solve(self.handle, a, b, o, int(iters), float(tol), ctypes.byref(st))
        if s not in (NS_OK, NS_NOT_CONVERGED):
            raise NSError(s, lib().ns_batch_last_error(self.handle).decode())
        return outs, s, st

    def result(self, i: int):
        st, it, sw = _int(), _int(), _int()
        rr = ctypes.c_double()
        lib().ns_batch_result(self.handle, i, ctypes.byref(st), ctypes.byref(it), ctypes.byref(sw), ctypes.byref(rr))
        return {"status": st.value, "ns_iters": it.value, "sweeps": sw.value, "rel_res": rr.value}


class Server:
    """Continuous-batching server (``ns_server_*``).

    ``Server(mem_budget_bytes, max_requests, max_nrhs, order=4, **options)``;
    ``submit(A, B, Theta, iters, tol)`` returns a ticket (the tensors must stay
    alive until the request is done); ``tick()`` runs one scheduling tick on
    the calling thread, or ``start()`` / ``stop()`` run ticks on a background
    thread; ``poll(ticket)`` returns the request's ``ns_result`` as a dict."""

    def __init__(self, mem_budget_bytes: int, max_requests: int, max_nrhs: int, order: int = 4, stream=None,
                 **options):
        self.opt = default_options(**options)
        h = _vp()
        s = lib().ns_server_create(int(mem_budget_bytes), int(max_requests), int(max_nrhs), int(order),
                                   ctypes.byref(self.opt), ctypes.byref(h))
        if s != NS_OK:
            raise NSError(s, "ns_server_create")
        self.handle = h.value
        self._keep: dict[int, tuple] = {}
        if stream is not None:
            lib().ns_server_set_stream(self.handle, _stream_ptr(stream))

    def close(self):
        if getattr(self, "handle", None):
            lib().ns_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _err(self, s: int, what: str):
        raise NSError(s, f"{what}: {lib().ns_server_last_error(self.handle).decode()}")

    def submit(self, A: torch.Tensor, B: torch.Tensor, Theta: torch.Tensor, iters: int = 64,
               tol: float = 1e-10) -> int:
        n = A.shape[0]
        if A.shape != (n, n) or B.dim() != 2 or B.shape[0] != n or Theta.shape != B.shape:
            raise ValueError("A must be n x n, B and Theta n x nrhs")
        req = ns_request(n, B.shape[1], int(iters), float(tol), _ptr(A), _ptr(B), _ptr(Theta))
        t = ctypes.c_uint64()
        s = lib().ns_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if s != NS_OK:
            self._err(s, "ns_server_submit")
        self._keep[t.value] = (A, B, Theta)
        return t.value

    def poll(self, ticket: int) -> dict:
        r = ns_result()
        s = lib().ns_server_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r))
        if s != NS_OK:
            self._err(s, "ns_server_poll")
        return {k: getattr(r, k) for k, _ in ns_result._fields_}

    def release(self, ticket: int) -> None:
        s = lib().ns_server_release(self.handle, ctypes.c_uint64(ticket))
        if s != NS_OK:
            self._err(s, "ns_server_release")
        self._keep.pop(ticket, None)

    def tick(self) -> int:
        a = _int()
        s = lib().ns_server_tick(self.handle, ctypes.byref(a))
        if s != NS_OK:
            self._err(s, "ns_server_tick")
        return a.value

    def start(self) -> None:
        s = lib().ns_server_start(self.handle)
        if s != NS_OK:
            self._err(s, "ns_server_start")

    def stop(self) -> None:
        s = lib().ns_server_stop(self.handle)
        if s != NS_OK:
            self._err(s, "ns_server_stop")

    def stats(self) -> dict:
        st = ns_server_stats()
        lib().ns_server_get_stats(self.handle, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in ns_server_stats._fields_}
