"""Thin ctypes binding of ``libhsma.so`` (include/hsma.h), same names as the C ABI.

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  There is no CPU fallback; if the library has not been built, loading
this module raises ``RuntimeError``.

Pointers are plain integers (e.g. ``tensor.data_ptr()``); streams are raw
``cudaStream_t`` values (e.g. ``torch.cuda.current_stream().cuda_stream``).
Helpers at the end move column-major numpy arrays to and from torch CUDA
tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhsma.so")

R64, C128, R32_BF16, R64_IR, R32, C64 = 0, 1, 2, 3, 4, 5
NON_UNIT, UNIT = 0, 1
LEFT, RIGHT = 0, 1
LOWER, UPPER = 0, 1
NO_TRANS, TRANS, CONJ_TRANS = 0, 1, 2
PATH_AUTO, PATH_SMALL, PATH_BLOCKED = 0, 1, 2
OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_NO_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_CONVERGED, ERR_BUSY = range(1, 8)
DEVERR_BAD_SIZE, DEVERR_NULL_PTR, DEVERR_TIMEOUT, DEVERR_BAD_PIVOT = 0x1, 0x2, 0x4, 0x8
DEVERR_NOT_CONVERGED = 0x10
STATUS_NAMES = {0: "HSMA_OK", 1: "HSMA_ERR_INVALID_ARG", 2: "HSMA_ERR_UNSUPPORTED", 3: "HSMA_ERR_NO_MEMORY",
                4: "HSMA_ERR_CUDA", 5: "HSMA_ERR_TIMEOUT", 6: "HSMA_ERR_NOT_CONVERGED", 7: "HSMA_ERR_BUSY"}

# Every function include/hsma.h declares (checked by the tests against the header).
EXPORTS = ["hsma_status_string", "hsma_version", "hsma_trsm_llnn", "hsma_trsm_llnn_ex",
           "hsma_trsm_llnn_vbatched", "hsma_plan", "hsma_small_cost", "hsma_tuning_load", "hsma_gen_matrix",
           "hsma_trace_enable", "hsma_trace_read", "hsma_trace_launches", "hsma_trace_reset",
           "hsma_device_status", "hsma_gemm_bf16_update", "hsma_gemm_f64_emulated", "hsma_trsm_llnn_vbatched_noalloc",
           "hsma_trsm_llnn_vbatched_host", "hsma_trsm_llnn_vbatched_host_tp", "hsma_trsm", "hsma_trsm_vbatched",
           "hsma_check_wait_timeout",
           "hsma_getrs_vbatched", "hsma_potrs_vbatched", "hsma_getrs", "hsma_potrs",
           "hsma_server_create", "hsma_server_submit", "hsma_server_poll", "hsma_server_drain", "hsma_server_stats",
           "hsma_server_destroy"]


class HsmaError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


class Plan(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("nb", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("split_k", ctypes.c_int32), ("looking", ctypes.c_int32),
                ("panel_cols", ctypes.c_int32), ("reserved", ctypes.c_int32)]


TILE_64x64, TILE_128x16, TILE_128x8 = 1, 2, 3
SPLITK_AUTO, SPLITK_OFF = 1, 2
LOOK_RIGHT, LOOK_LEFT = 1, 2


class Opts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("nb", ctypes.c_int32), ("groups", ctypes.c_int32),
                ("ir_max_iter", ctypes.c_int32), ("ir_tol", ctypes.c_double), ("bf16_terms", ctypes.c_int32),
                ("ir_residual", ctypes.c_int32), ("fp64_products", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("split_k", ctypes.c_int32), ("looking", ctypes.c_int32), ("panel_cols", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("diag", ctypes.c_int32), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("alpha", ctypes.c_double * 2), ("A_host", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B_host", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("gen_seed", ctypes.c_uint64),
                ("gen_inst", ctypes.c_int64), ("X_host", ctypes.c_void_p), ("ldx", ctypes.c_int64),
                ("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ipiv_host", ctypes.c_void_p)]


REQ_TRSM, REQ_GETRS, REQ_POTRS = 0, 1, 2


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "admitted", "completed", "bytes_in_use",
                                               "peak_bytes_in_use", "budget_bytes", "batched_launches",
                                               "blocked_launches")]


SERVER_FAKE_DEVICE = 0x1
SERVER_FP64_EMULATED = 0x2


class Info(ctypes.Structure):
    _fields_ = [("plan", Plan), ("ir_iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("ir_residual", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhsma.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                           "python paper_2608_25469_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, u32p, vp, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double
    c_int = ctypes.c_int
    lib.hsma_status_string.argtypes = [c_int]
    lib.hsma_status_string.restype = ctypes.c_char_p
    lib.hsma_version.restype = ctypes.c_char_p
    lib.hsma_trsm_llnn.argtypes = [c_int, c_int, i64, i64, vp, vp, i64, vp, i64, vp]
    lib.hsma_trsm_llnn.restype = c_int
    lib.hsma_trsm_llnn_ex.argtypes = [c_int, c_int, i64, i64, vp, vp, i64, vp, i64, vp,
                                      ctypes.POINTER(Opts), ctypes.POINTER(Info)]
    lib.hsma_trsm_llnn_ex.restype = c_int
    lib.hsma_trsm_llnn_vbatched.argtypes = [c_int, c_int, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, u32p, vp]
    lib.hsma_trsm_llnn_vbatched.restype = c_int
    lib.hsma_trsm_llnn_vbatched_noalloc.argtypes = [c_int, c_int, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, u32p,
                                                    vp]
    lib.hsma_trsm_llnn_vbatched_noalloc.restype = c_int
    lib.hsma_trsm_llnn_vbatched_host.argtypes = [c_int, c_int, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    lib.hsma_trsm_llnn_vbatched_host.restype = c_int
    lib.hsma_trsm_llnn_vbatched_host_tp.argtypes = [c_int, c_int, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    lib.hsma_trsm_llnn_vbatched_host_tp.restype = c_int
    lib.hsma_trsm.argtypes = [c_int, c_int, c_int, c_int, c_int, i64, i64, vp, vp, i64, vp, i64, vp, vp, vp]
    lib.hsma_trsm.restype = c_int
    lib.hsma_trsm_vbatched.argtypes = [c_int, c_int, c_int, c_int, c_int, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32,
                                       u32p, vp]
    lib.hsma_trsm_vbatched.restype = c_int
    lib.hsma_plan.argtypes = [c_int, i64, i64, ctypes.POINTER(Plan)]
    lib.hsma_plan.restype = c_int
    lib.hsma_small_cost.argtypes = [c_int, i64, i64, i32]
    lib.hsma_small_cost.restype = dbl
    lib.hsma_tuning_load.argtypes = [ctypes.c_char_p]
    lib.hsma_tuning_load.restype = c_int
    lib.hsma_gen_matrix.argtypes = [c_int, c_int, ctypes.c_uint64, i64, i64, i64, vp, i64, vp]
    lib.hsma_gen_matrix.restype = c_int
    lib.hsma_trace_enable.argtypes = [c_int]
    lib.hsma_trace_enable.restype = c_int
    lib.hsma_trace_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_longlong)]
    lib.hsma_trace_read.restype = c_int
    lib.hsma_trace_launches.restype = ctypes.c_longlong
    lib.hsma_trace_reset.restype = None
    lib.hsma_gemm_bf16_update.argtypes = [i64, i64, i64, vp, vp, ctypes.c_float, vp, i64, vp]
    lib.hsma_gemm_bf16_update.restype = c_int
    lib.hsma_gemm_f64_emulated.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp]
    lib.hsma_gemm_f64_emulated.restype = c_int
    lib.hsma_server_create.argtypes = [ctypes.c_size_t, c_int, ctypes.c_uint, ctypes.POINTER(ctypes.c_void_p)]
    lib.hsma_server_create.restype = c_int
    lib.hsma_server_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.hsma_server_submit.restype = c_int
    lib.hsma_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(c_int), ctypes.POINTER(dbl)]
    lib.hsma_server_poll.restype = c_int
    lib.hsma_server_drain.argtypes = [vp, dbl]
    lib.hsma_server_drain.restype = c_int
    lib.hsma_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.hsma_server_stats.restype = c_int
    lib.hsma_server_destroy.argtypes = [vp]
    lib.hsma_server_destroy.restype = c_int
    lib.hsma_device_status.argtypes = [ctypes.POINTER(ctypes.c_uint)]
    lib.hsma_device_status.restype = c_int
    lib.hsma_getrs_vbatched.argtypes = [c_int, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, u32p, vp]
    lib.hsma_getrs_vbatched.restype = c_int
    lib.hsma_potrs_vbatched.argtypes = [c_int, i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, u32p, vp]
    lib.hsma_potrs_vbatched.restype = c_int
    lib.hsma_getrs.argtypes = [c_int, i64, i64, vp, vp, i64, vp, vp, i64, vp, ctypes.POINTER(Opts)]
    lib.hsma_getrs.restype = c_int
    lib.hsma_potrs.argtypes = [c_int, i64, i64, vp, vp, i64, vp, i64, vp, ctypes.POINTER(Opts)]
    lib.hsma_potrs.restype = c_int
    lib.hsma_check_wait_timeout.argtypes = [ctypes.c_uint64, vp, vp]
    lib.hsma_check_wait_timeout.restype = c_int
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def _check(status: int, where: str):
    if status != OK:
        raise HsmaError(status, where)


def _alpha_buf(alpha):
    a = complex(alpha)
    return (ctypes.c_double * 2)(a.real, a.imag)


def hsma_status_string(status: int) -> str:
    return _lib.hsma_status_string(status).decode()


def hsma_version() -> str:
    return _lib.hsma_version().decode()


def hsma_trsm_llnn(dtype, diag, m, n, alpha, A, lda, B, ldb, stream=0, check=True) -> int:
    """Raw call; A and B are device pointers (ints).  Returns the status."""
    s = _lib.hsma_trsm_llnn(dtype, diag, m, n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), A, lda, B, ldb,
                            stream)
    if check:
        _check(s, "hsma_trsm_llnn")
    return s


def hsma_trsm_llnn_ex(dtype, diag, m, n, alpha, A, lda, B, ldb, stream=0, opts: Opts | None = None,
                      info: Info | None = None, check=True) -> int:
    s = _lib.hsma_trsm_llnn_ex(dtype, diag, m, n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), A, lda, B, ldb,
                               stream, ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(info) if info is not None else None)
    if check:
        _check(s, "hsma_trsm_llnn_ex")
    return s


def hsma_trsm(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream=0, opts: Opts | None = None,
              info: Info | None = None, check=True) -> int:
    """BLAS triangular-solve variants: side LEFT/RIGHT, uplo LOWER/UPPER, trans NO_TRANS/TRANS/CONJ_TRANS."""
    s = _lib.hsma_trsm(dtype, side, uplo, trans, diag, m, n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), A,
                       lda, B, ldb, stream, ctypes.byref(opts) if opts is not None else None,
                       ctypes.byref(info) if info is not None else None)
    if check:
        _check(s, "hsma_trsm")
    return s


def hsma_trsm_vbatched(dtype, side, uplo, trans, diag, batch, d_m, d_n, alpha, d_A, d_lda, d_B, d_ldb, max_m=0,
                       max_n=0, d_status=0, stream=0, check=True) -> int:
    """Varlen batch of left-side variants (uplo, trans) with in-kernel index remapping."""
    s = _lib.hsma_trsm_vbatched(dtype, side, uplo, trans, diag, batch, d_m, d_n,
                                ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), d_A, d_lda, d_B, d_ldb, max_m, max_n,
                                d_status or None, stream)
    if check:
        _check(s, "hsma_trsm_vbatched")
    return s


def hsma_getrs_vbatched(dtype, batch, d_m, d_n, alpha, d_LU, d_lda, d_ipiv, d_B, d_ldb, max_m=0, max_n=0,
                        d_status=0, stream=0, check=True) -> int:
    """Varlen batch of LU-factor solves in one launch: X = U^{-1} L^{-1} P^T (alpha B) per instance
    (packed getrf factors; d_ipiv: device array of per-instance pivot pointers, or 0 for none)."""
    s = _lib.hsma_getrs_vbatched(dtype, batch, d_m, d_n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), d_LU,
                                 d_lda, d_ipiv or None, d_B, d_ldb, max_m, max_n, d_status or None, stream)
    if check:
        _check(s, "hsma_getrs_vbatched")
    return s


def hsma_getrs(dtype, m, n, alpha, LU, lda, ipiv, B, ldb, stream=0, opts: Opts | None = None, check=True) -> int:
    """One solve from LU factors (device pointers; ipiv: device int32 pivots or 0)."""
    s = _lib.hsma_getrs(dtype, m, n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), LU, lda, ipiv or None, B, ldb,
                        stream or None, ctypes.byref(opts) if opts is not None else None)
    if check:
        _check(s, "hsma_getrs")
    return s


def hsma_potrs(dtype, m, n, alpha, L, lda, B, ldb, stream=0, opts: Opts | None = None, check=True) -> int:
    """One solve from a lower Cholesky factor (device pointers)."""
    s = _lib.hsma_potrs(dtype, m, n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), L, lda, B, ldb,
                        stream or None, ctypes.byref(opts) if opts is not None else None)
    if check:
        _check(s, "hsma_potrs")
    return s


def hsma_potrs_vbatched(dtype, batch, d_m, d_n, alpha, d_L, d_lda, d_B, d_ldb, max_m=0, max_n=0, d_status=0,
                        stream=0, check=True) -> int:
    """Varlen batch of Cholesky-factor solves in one launch: X = L^{-H} L^{-1} (alpha B) per instance."""
    s = _lib.hsma_potrs_vbatched(dtype, batch, d_m, d_n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), d_L,
                                 d_lda, d_B, d_ldb, max_m, max_n, d_status or None, stream)
    if check:
        _check(s, "hsma_potrs_vbatched")
    return s


def hsma_trsm_llnn_vbatched(dtype, diag, batch, d_m, d_n, alpha, d_A, d_lda, d_B, d_ldb, max_m=0, max_n=0,
                            d_status=0, stream=0, check=True) -> int:
    s = _lib.hsma_trsm_llnn_vbatched(dtype, diag, batch, d_m, d_n, ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p),
                                     d_A, d_lda, d_B, d_ldb, max_m, max_n, d_status or None, stream)
    if check:
        _check(s, "hsma_trsm_llnn_vbatched")
    return s


def hsma_trsm_llnn_vbatched_noalloc(dtype, diag, batch, d_m, d_n, alpha, d_A, d_lda, d_B, d_ldb, max_m=0,
                                    max_n=0, d_status=0, stream=0, check=True) -> int:
    """Allocation-free varlen batch: schedule scratch in a static device array (batch <= 65536)."""
    s = _lib.hsma_trsm_llnn_vbatched_noalloc(dtype, diag, batch, d_m, d_n,
                                             ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), d_A, d_lda, d_B,
                                             d_ldb, max_m, max_n, d_status or None, stream)
    if check:
        _check(s, "hsma_trsm_llnn_vbatched_noalloc")
    return s


def hsma_trsm_llnn_vbatched_host(dtype, diag, batch, h_m, h_n, alpha, hA, h_offA, hB, h_offB, hX, chunks=0,
                                 stream=0, check=True) -> int:
    """Varlen batch with matrices in host memory (pointers as ints; h_m, h_n int32 and h_offA,
    h_offB int64 host arrays, numpy arrays accepted), copies overlapped with the solves."""
    def ptr(a):
        return a.ctypes.data if isinstance(a, np.ndarray) else a
    s = _lib.hsma_trsm_llnn_vbatched_host(dtype, diag, batch, ptr(h_m), ptr(h_n),
                                          ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), ptr(hA), ptr(h_offA),
                                          ptr(hB), ptr(h_offB), ptr(hX), chunks, stream)
    if check:
        _check(s, "hsma_trsm_llnn_vbatched_host")
    return s


def hsma_trsm_llnn_vbatched_host_tp(dtype, diag, batch, h_m, h_n, alpha, hAp, h_offA, hB, h_offB, hX, chunks=0,
                                    stream=0, check=True) -> int:
    """As hsma_trsm_llnn_vbatched_host with each A_i as a packed lower triangle in host memory."""
    def ptr(a):
        return a.ctypes.data if isinstance(a, np.ndarray) else a
    s = _lib.hsma_trsm_llnn_vbatched_host_tp(dtype, diag, batch, ptr(h_m), ptr(h_n),
                                             ctypes.cast(_alpha_buf(alpha), ctypes.c_void_p), ptr(hAp), ptr(h_offA),
                                             ptr(hB), ptr(h_offB), ptr(hX), chunks, stream)
    if check:
        _check(s, "hsma_trsm_llnn_vbatched_host_tp")
    return s


def hsma_server_create(budget_bytes: int, n_streams: int = 4, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(_lib.hsma_server_create(budget_bytes, n_streams, flags, ctypes.byref(h)), "hsma_server_create")
    return h.value


def hsma_server_submit(server: int, req: Request) -> int:
    t = ctypes.c_uint64()
    _check(_lib.hsma_server_submit(server, ctypes.byref(req), ctypes.byref(t)), "hsma_server_submit")
    return t.value


def hsma_server_poll(server: int, ticket: int):
    """(done, latency_s, status) of a request."""
    d = ctypes.c_int()
    lat = ctypes.c_double()
    s = _lib.hsma_server_poll(server, ticket, ctypes.byref(d), ctypes.byref(lat))
    return bool(d.value), lat.value, s


def hsma_server_drain(server: int, timeout_s: float = 0.0) -> int:
    return _lib.hsma_server_drain(server, timeout_s)


def hsma_server_stats(server: int) -> ServerStats:
    st = ServerStats()
    _check(_lib.hsma_server_stats(server, ctypes.byref(st)), "hsma_server_stats")
    return st


def hsma_server_destroy(server: int) -> int:
    return _lib.hsma_server_destroy(server)


def hsma_plan(dtype, m, n) -> Plan:
    p = Plan()
    _check(_lib.hsma_plan(dtype, m, n, ctypes.byref(p)), "hsma_plan")
    return p


def hsma_small_cost(dtype, m, n, groups) -> float:
    return _lib.hsma_small_cost(dtype, m, n, groups)


def hsma_tuning_load(path: str | None) -> int:
    return _lib.hsma_tuning_load(path.encode() if path is not None else None)


def hsma_gen_matrix(dtype, kind, seed, inst, m, cols, dst, ld, stream=0, check=True) -> int:
    s = _lib.hsma_gen_matrix(dtype, kind, seed, inst, m, cols, dst, ld, stream)
    if check:
        _check(s, "hsma_gen_matrix")
    return s


def hsma_gemm_bf16_update(M, N, K, A, Bt, beta, C, ldc, stream=0, check=True) -> int:
    s = _lib.hsma_gemm_bf16_update(M, N, K, A, Bt, beta, C, ldc, stream)
    if check:
        _check(s, "hsma_gemm_bf16_update")
    return s


def hsma_gemm_f64_emulated(M, N, K, A, lda, X, ldx, C, ldc, stream=0, check=True) -> int:
    """C -= A X in FP64 emulated on the BF16 tensor cores (device pointers, column-major)."""
    s = _lib.hsma_gemm_f64_emulated(M, N, K, A, lda, X, ldx, C, ldc, stream)
    if check:
        _check(s, "hsma_gemm_f64_emulated")
    return s


def hsma_device_status() -> int:
    """Device error bits raised since the last call (synchronises the device)."""
    v = ctypes.c_uint()
    _check(_lib.hsma_device_status(ctypes.byref(v)), "hsma_device_status")
    return v.value


def hsma_check_wait_timeout(limit_ns: int, d_returned: int, stream: int = 0, check: bool = True) -> int:
    """Launch the self-check whose bounded wait runs out after limit_ns (device int at d_returned)."""
    s = _lib.hsma_check_wait_timeout(int(limit_ns), d_returned or None, stream or None)
    if check:
        _check(s, "hsma_check_wait_timeout")
    return s


def hsma_trace_enable(on: bool) -> int:
    return _lib.hsma_trace_enable(int(bool(on)))


def hsma_trace_read(phase: str):
    """(total device ms, launch count) of a traced phase since the last reset."""
    ms = ctypes.c_double()
    cnt = ctypes.c_longlong()
    _check(_lib.hsma_trace_read(phase.encode(), ctypes.byref(ms), ctypes.byref(cnt)), "hsma_trace_read")
    return ms.value, cnt.value


def hsma_trace_launches() -> int:
    return _lib.hsma_trace_launches()


def hsma_trace_reset() -> None:
    _lib.hsma_trace_reset()


# ---------------------------------------------------------------------------
# Column-major helpers (torch only moves memory).
# ---------------------------------------------------------------------------
def to_device(X: np.ndarray, device="cuda"):
    """Fortran-ordered (ld, cols) numpy array -> CUDA tensor with the same column-major bytes.

    The tensor has shape (cols, ld) in torch's row-major convention."""
    import torch
    Xf = np.asfortranarray(X)
    return torch.from_numpy(np.ascontiguousarray(Xf.T)).to(device)


def from_device(t) -> np.ndarray:
    """Inverse of ``to_device``: returns a Fortran-ordered (ld, cols) numpy array."""
    return np.asfortranarray(t.cpu().numpy().T)


def stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)
