"""Thin ctypes binding of libbse_gb300.so (the C ABI in include/bse.h and
include/bse_stages.h). Argument marshalling only: every step of the solver runs
in the library's CUDA kernels. Loading fails loudly if the library has not been
built (``python -m paper_1501_03830_gb300.build``); there is no fallback.

Array arguments may be numpy arrays (host memory) or torch tensors (host or
CUDA). Complex matrices are complex128, column-major (Fortran order).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbse_gb300.so")

BSE_OK = 0
BSE_ERR_ARG = -1
BSE_ERR_NOT_DEFINITE = -2
BSE_ERR_NOT_CONVERGED = -3
BSE_ERR_NOMEM = -4
BSE_ERR_BUSY = -5
BSE_ERR_TIMEOUT = -6
BSE_ERR_CUDA = -7
BSE_ERR_NO_TICKET = -8

BSE_FP64 = 0
BSE_MIXED = 1
BSE_MIXED_REFINED = 2

PRECISIONS = {"fp64": BSE_FP64, "mixed": BSE_MIXED, "mixed_refined": BSE_MIXED_REFINED}

STAGE_NAMES = ["form_M", "cholesky", "form_W", "tridiag", "tdeig", "backtransform", "refine", "weights", "copies",
               "total"]

# Every symbol the headers declare (checked by the CPU test suite).
EXPORTS = [
    "bse_create", "bse_destroy", "bse_set_stream", "bse_set_timing", "bse_solve", "bse_solve_real", "bse_spectrum",
    "bse_absorption",
    "bse_sol_view",
    "bse_sol_free", "bse_serve_start", "bse_submit", "bse_poll", "bse_serve_stop", "bse_solve_batched",
    "bse_last_error", "bse_version", "bse_launch_count", "bse_kprof_enable", "bse_kprof_read",
    "bse_stage_form_M", "bse_stage_potrf_worksize", "bse_stage_potrf", "bse_stage_form_W",
    "bse_stage_tridiag_worksize", "bse_stage_tridiag", "bse_debug_trace_tridiag", "bse_debug_barrier_spin", "bse_stage_tridiag_grid", "bse_stage_tdeig_worksize", "bse_stage_tdeig", "bse_stage_tdeig_noalloc",
    "bse_stage_backtransform_worksize", "bse_stage_backtransform", "bse_stage_weights", "bse_stage_broaden",
    "bse_stage_refine_worksize", "bse_stage_refine", "bse_tc_gemm_bf16", "bse_ozaki_worksize", "bse_ozaki_gemm",
    "bse_ozaki_digit_bits",
    "bse_tc32_gemm", "bse_set_fp32_gemm",
    "bse_stage_sbr_worksize", "bse_stage_sbr", "bse_stage_sbr_apply_q2", "bse_stage_sbr_backtransform",
    "bse_set_band_reduction", "bse_stage_tdeig_reorth_worksize", "bse_stage_tdeig_reorth",
    "bse_stage_tdeig_mrrr_worksize", "bse_stage_tdeig_mrrr", "bse_set_tdeig_method",
]


class BSEError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str = ""):
        super().__init__(f"{where}: status {code} {msg}".strip())
        self.code = code


class bse_info(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("info", C.c_int), ("precision", C.c_int), ("sweeps", C.c_int),
        ("stage_ms", C.c_double * 10), ("refine_resid", C.c_double), ("refine_dlam", C.c_double),
        ("unrefined_dlam", C.c_double),
    ]


class bse_request(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("A", C.c_void_p), ("B", C.c_void_p), ("d_r", C.c_void_p), ("d_l", C.c_void_p),
        ("precision", C.c_int), ("lambda_", C.c_void_p), ("X", C.c_void_p), ("w", C.c_void_p),
    ]


class bse_result(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("n", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
        ("t_done", C.c_double), ("refine_dlam", C.c_double),
    ]


_lib = None


def lib() -> C.CDLL:
    """Load the library (once). Raises if it is missing: there is no CPU path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1501_03830_gb300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "bse_create": (i, [C.POINTER(vp), i, sz]),
        "bse_destroy": (i, [vp]),
        "bse_set_stream": (i, [vp, vp]),
        "bse_set_timing": (i, [vp, i]),
        "bse_solve": (i, [vp, i, vp, i, vp, i, i, vp, vp, vp, C.POINTER(vp), C.POINTER(bse_info)]),
        "bse_solve_real": (i, [vp, i, vp, i, vp, i, i, vp, vp, vp, C.POINTER(bse_info)]),
        "bse_spectrum": (i, [vp, vp, vp, vp, vp]),
        "bse_absorption": (i, [vp, vp, vp, vp, i, vp, C.c_double, vp, vp]),
        "bse_sol_view": (i, [vp, C.POINTER(i), C.POINTER(vp), C.POINTER(vp)]),
        "bse_sol_free": (i, [vp]),
        "bse_serve_start": (i, [vp, i]),
        "bse_submit": (i, [vp, C.POINTER(bse_request), C.POINTER(C.c_uint64)]),
        "bse_poll": (i, [vp, C.c_uint64, C.POINTER(bse_result), C.POINTER(i)]),
        "bse_serve_stop": (i, [vp, d]),
        "bse_solve_batched": (i, [vp, i, vp, vp, vp, i, vp, vp, vp]),
        "bse_launch_count": (C.c_longlong, []),
        "bse_kprof_enable": (i, [i]),
        "bse_kprof_read": (i, [i, C.POINTER(C.c_longlong), C.POINTER(d), C.POINTER(d), C.POINTER(d)]),
        "bse_last_error": (C.c_char_p, []),
        "bse_version": (C.c_char_p, []),
        "bse_stage_form_M": (i, [i, vp, i, vp, i, vp, i, vp, i, vp]),
        "bse_stage_potrf_worksize": (sz, [i, i]),
        "bse_stage_potrf": (i, [i, vp, i, i, vp, vp, vp]),
        "bse_stage_form_W": (i, [i, vp, i, vp, i, i, vp]),
        "bse_stage_tridiag_worksize": (sz, [i, i]),
        "bse_stage_tridiag": (i, [i, vp, i, vp, vp, i, vp, vp, vp]),
        "bse_debug_trace_tridiag": (i, [vp, i]),
        "bse_debug_barrier_spin": (i, [C.c_long]),
        "bse_stage_tridiag_grid": (i, [i, i]),
        "bse_stage_tdeig_worksize": (sz, [i]),
        "bse_stage_tdeig": (i, [i, vp, vp, vp, vp, vp, vp]),
        "bse_stage_tdeig_noalloc": (i, [i, vp, vp, vp, vp, vp]),
        "bse_stage_backtransform_worksize": (sz, [i, i]),
        "bse_stage_backtransform": (i, [i, vp, i, vp, i, vp, vp, vp, vp, vp, i, i, vp, vp]),
        "bse_stage_weights": (i, [i, vp, i, vp, vp, vp, vp]),
        "bse_stage_broaden": (i, [i, vp, vp, i, vp, C.c_double, vp, vp, vp]),
        "bse_stage_refine_worksize": (sz, [i]),
        "bse_stage_refine": (i, [i, vp, vp, vp, i, vp, vp, vp, C.POINTER(i), C.POINTER(d)]),
        "bse_tc_gemm_bf16": (i, [i, i, i, vp, vp, i, vp, i, vp, vp]),
        "bse_ozaki_worksize": (sz, [i, i, i, i]),
        "bse_ozaki_digit_bits": (i, [i]),
        "bse_ozaki_gemm": (i, [i, i, i, vp, i, vp, i, vp, i, i, vp, vp, vp]),
        "bse_tc32_gemm": (i, [i, i, i, C.c_float, vp, i, i, vp, i, i, C.c_float, vp, i, i, i, vp, vp]),
        "bse_set_fp32_gemm": (i, [i]),
        "bse_stage_sbr_worksize": (sz, [i]),
        "bse_stage_sbr": (i, [i, vp, i, vp, vp, vp, vp, vp]),
        "bse_stage_sbr_apply_q2": (i, [i, vp, i, vp, vp]),
        "bse_stage_sbr_backtransform": (i, [i, vp, i, vp, i, vp, vp, vp, vp, vp, i, vp, vp, vp]),
        "bse_set_band_reduction": (i, [i]),
        "bse_stage_tdeig_reorth_worksize": (sz, [i]),
        "bse_stage_tdeig_reorth": (i, [i, vp, vp, vp]),
        "bse_stage_tdeig_mrrr_worksize": (sz, [i, i, i]),
        "bse_stage_tdeig_mrrr": (i, [i, vp, vp, i, i, i, d, vp, vp, i, i, vp, vp, vp]),
        "bse_set_tdeig_method": (i, [i]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return lib().bse_last_error().decode()


def check(rc: int, where: str) -> None:
    if rc != BSE_OK:
        raise BSEError(rc, where, last_error())


def ptr(a) -> int | None:
    """Raw address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"cannot take the address of {type(a)}")


def _fortran_c128(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.complex128))


class Solution:
    """A device-resident solution kept by bse_solve (for bse_spectrum)."""

    def __init__(self, handle: int):
        self.handle = C.c_void_p(handle)

    def view(self):
        n = C.c_int()
        lam = C.c_void_p()
        X = C.c_void_p()
        check(lib().bse_sol_view(self.handle, C.byref(n), C.byref(lam), C.byref(X)), "bse_sol_view")
        return n.value, lam.value, X.value

    def free(self) -> None:
        if self.handle:
            lib().bse_sol_free(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """bse_create / bse_destroy around one GPU."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        h = C.c_void_p()
        check(lib().bse_create(C.byref(h), device, hbm_budget), "bse_create")
        self.handle = h

    def close(self) -> None:
        if self.handle:
            lib().bse_destroy(self.handle)
            self.handle = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle: int | None) -> None:
        check(lib().bse_set_stream(self.handle, stream_handle), "bse_set_stream")

    def set_timing(self, on: bool) -> None:
        check(lib().bse_set_timing(self.handle, int(on)), "bse_set_timing")

    def solve(self, A, B, precision="fp64", want_X=True, want_Y=False, keep=False, out=None):
        """bse_solve on host (numpy) or device (torch) inputs.

        Host inputs give host outputs (numpy); with ``out`` = dict of torch tensors
        (lambda, X, Y) the results go there instead. Returns (lam, X, Y, info, sol).
        """
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if isinstance(A, np.ndarray):
            A = _fortran_c128(A)
            B = _fortran_c128(B)
            n = A.shape[0]
            lda = A.shape[0]
            ldb = B.shape[0]
        else:
            n = A.shape[-1]
            lda = n
            ldb = n
        m = 2 * n
        if out is not None:
            lam, X, Y = out.get("lambda"), out.get("X"), out.get("Y")
        else:
            lam = np.empty(n, dtype=np.float64)
            X = np.empty((m, n), dtype=np.complex128, order="F") if want_X else None
            Y = np.empty((m, n), dtype=np.complex128, order="F") if want_Y else None
        info = bse_info()
        solh = C.c_void_p()
        rc = lib().bse_solve(self.handle, n, ptr(A), lda, ptr(B), ldb, prec, ptr(lam), ptr(X), ptr(Y),
                             C.byref(solh) if keep else None, C.byref(info))
        check(rc, "bse_solve")
        sol = Solution(solh.value) if keep else None
        return lam, X, Y, info, sol

    def solve_real(self, A, B, precision="fp64", want_X=True, out=None):
        """bse_solve_real (Algorithm 2) on real symmetric A, B (numpy host or torch
        device, n x n FP64). Returns (lam, X1, X2, info); host inputs give numpy
        outputs, ``out`` = dict of torch tensors (lambda, X1, X2) receives them
        instead."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if isinstance(A, np.ndarray):
            A = np.asfortranarray(A, dtype=np.float64)
            B = np.asfortranarray(B, dtype=np.float64)
        n = A.shape[-1]
        if out is not None:
            lam, X1, X2 = out.get("lambda"), out.get("X1"), out.get("X2")
        else:
            lam = np.empty(n, dtype=np.float64)
            X1 = np.empty((n, n), dtype=np.float64, order="F") if want_X else None
            X2 = np.empty((n, n), dtype=np.float64, order="F") if want_X else None
        info = bse_info()
        rc = lib().bse_solve_real(self.handle, n, ptr(A), n, ptr(B), n, prec, ptr(lam), ptr(X1), ptr(X2),
                                  C.byref(info))
        check(rc, "bse_solve_real")
        return lam, X1, X2, info

    def spectrum(self, sol: Solution, d_r, d_l, out=None):
        """bse_spectrum: complex weights of Eq. absp."""
        if isinstance(d_r, np.ndarray):
            d_r = np.ascontiguousarray(d_r, dtype=np.complex128)
            d_l = np.ascontiguousarray(d_l, dtype=np.complex128)
        n, _, _ = sol.view()
        w = out if out is not None else np.empty(n, dtype=np.complex128)
        check(lib().bse_spectrum(self.handle, sol.handle, ptr(d_r), ptr(d_l), ptr(w)), "bse_spectrum")
        return w

    def absorption(self, sol: Solution, omega, sigma: float, d_r=None, d_l=None, out=None):
        """bse_absorption: Gaussian-broadened spectral density (Eq. DOS) and, with
        dipoles, absorption spectrum (Eq. absp) on the grid ``omega``. Returns
        (dos, eps) with eps None without dipoles; numpy in, numpy out unless
        ``out`` = (dos, eps) device buffers are given."""
        if isinstance(omega, np.ndarray):
            omega = np.ascontiguousarray(omega, dtype=np.float64)
        if isinstance(d_r, np.ndarray):
            d_r = np.ascontiguousarray(d_r, dtype=np.complex128)
            d_l = np.ascontiguousarray(d_l, dtype=np.complex128)
        k = len(omega)
        if out is not None:
            dos, eps = out
        else:
            dos = np.empty(k, dtype=np.float64)
            eps = np.empty(k, dtype=np.complex128) if d_r is not None else None
        check(lib().bse_absorption(self.handle, sol.handle, ptr(d_r), ptr(d_l), k, ptr(omega), float(sigma), ptr(dos),
                                   ptr(eps)), "bse_absorption")
        return dos, eps

    def solve_batched(self, problems, precision="mixed_refined", want_X=True, outs=None):
        """bse_solve_batched over a list of (A, B) pairs (numpy host arrays or
        device tensors, each n x n complex128). Results go to ``outs`` (a list of
        (lambda, X) buffers, X may be None) or to new host arrays. Returns
        (list of (lambda, X), per-problem status array)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        count = len(problems)
        keep = []  # holds the marshalled inputs alive for the call
        ns = (C.c_int * count)()
        pa = (C.c_void_p * count)()
        pb = (C.c_void_p * count)()
        pl = (C.c_void_p * count)()
        px = (C.c_void_p * count)()
        results = []
        for i, (A, B) in enumerate(problems):
            if isinstance(A, np.ndarray):
                A = _fortran_c128(A)
                B = _fortran_c128(B)
                n = A.shape[0]
            else:
                n = A.shape[-1]
            keep.append((A, B))
            if outs is not None:
                lam, X = outs[i]
            else:
                lam = np.empty(n, dtype=np.float64)
                X = np.empty((2 * n, n), dtype=np.complex128, order="F") if want_X else None
            results.append((lam, X))
            ns[i], pa[i], pb[i], pl[i], px[i] = n, ptr(A), ptr(B), ptr(lam), ptr(X)
        st = (C.c_int * count)()
        rc = lib().bse_solve_batched(self.handle, count, ns, pa, pb, prec, pl, px, st)
        if rc != 0 and not any(st):  # a call-level failure (per-problem ones are in the statuses)
            check(rc, "bse_solve_batched")
        return results, np.array(list(st), dtype=np.int32)

    # --- request loop ---------------------------------------------------------
    def serve_start(self, slots: int = 2) -> None:
        check(lib().bse_serve_start(self.handle, slots), "bse_serve_start")

    def submit(self, req: bse_request) -> int:
        t = C.c_uint64()
        check(lib().bse_submit(self.handle, C.byref(req), C.byref(t)), "bse_submit")
        return t.value

    def submit_rc(self, req: bse_request) -> tuple[int, int]:
        t = C.c_uint64()
        rc = lib().bse_submit(self.handle, C.byref(req), C.byref(t))
        return rc, t.value

    def poll(self, ticket: int):
        res = bse_result()
        done = C.c_int()
        check(lib().bse_poll(self.handle, ticket, C.byref(res), C.byref(done)), "bse_poll")
        return bool(done.value), res

    def serve_stop(self, timeout_s: float = 600.0) -> int:
        return lib().bse_serve_stop(self.handle, timeout_s)


def make_request(n, A, B, lam, X=None, d_r=None, d_l=None, w=None, precision="mixed_refined") -> bse_request:
    """A request for bse_submit. numpy inputs are laid out column-major here; the
    request keeps references to every buffer it points to, so they live as long
    as the request object (keep it until bse_poll reports it done)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if isinstance(A, np.ndarray):
        A = _fortran_c128(A)
        B = _fortran_c128(B)
    if isinstance(d_r, np.ndarray):
        d_r = np.ascontiguousarray(d_r, dtype=np.complex128)
        d_l = np.ascontiguousarray(d_l, dtype=np.complex128)
    r = bse_request()
    r._keep = (A, B, lam, X, d_r, d_l, w)
    r.n = n
    r.A, r.B = ptr(A), ptr(B)
    r.d_r, r.d_l = ptr(d_r), ptr(d_l)
    r.precision = prec
    r.lambda_ = ptr(lam)
    r.X = ptr(X)
    r.w = ptr(w)
    return r


KPROF_CLASSES = ["form_M", "potrf_diag", "gemm_f64", "gemm_f32", "trd_symv", "trd_col", "tdeig_bisect",
                 "tdeig_vec", "weights", "elementwise", "gemm_tc", "gemm_tf32", "sbr_qr", "sbr_chase", "sbr_q2",
                 "tf32_split"]


def launch_count() -> int:
    return int(lib().bse_launch_count())


def kprof_enable(on: bool) -> None:
    check(lib().bse_kprof_enable(int(on)), "bse_kprof_enable")


def kprof_read() -> dict:
    """Per kernel class: launches, device ms, charged bytes and flops."""
    out = {}
    for k, name in enumerate(KPROF_CLASSES):
        n = C.c_longlong()
        ms, b, f = C.c_double(), C.c_double(), C.c_double()
        check(lib().bse_kprof_read(k, C.byref(n), C.byref(ms), C.byref(b), C.byref(f)), "bse_kprof_read")
        out[name] = {"launches": n.value, "ms": ms.value, "bytes": b.value, "flops": f.value}
    return out


def version() -> str:
    return lib().bse_version().decode()
