"""Oracle for the triangular solve L X = alpha B (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may import this package.  The library itself never does: it has no
CPU fallback.  The arithmetic lives in ``trsm_oracle.c`` (plain C, fp64 and
complex128, compiled with ``-O2 -ffp-contract=off``); this module compiles it
on first use and wraps it with ctypes.

Every function cites the passage it follows:

* ``solve``, ``solve_cols``, ``solve_batch``: the forward-substitution formula of
  Section 2.1 (repeated in Section 4.2.1),
  x_ij = (alpha b_ij - sum_{k<i} a_ik x_kj) / a_ii, columns independent.
* ``backward_error``: normwise backward error with a compensated residual (the
  acceptance measure for the solve; Frobenius norms as in Table 2's metric).
* ``forward_error``: normwise relative forward error ||X - X_ref||_F / ||X_ref||_F,
  the measure of Table 2.
* ``solve_general``: the BLAS variants (side, uplo, trans, diag) by definition.
* ``getrs``: the solve from LU factors (Section 1's motivating use): row
  interchanges in order, then the unit-lower and the upper solve.
* ``potrs``: the solve from a lower Cholesky factor: the lower solve, then
  the conjugate-transposed one.

Pins (see ``tests/test_oracle_pins.py``): identity and diagonal A, the unit
lower-bidiagonal closed form, exact rational elimination on small dyadic inputs,
LAPACK's triangular solve, the backward-error bound, and invariants (upper
triangle never read, unit diagonal never read, columns independent, complex with
zero imaginary part equals real).  ``getrs`` is pinned in
``tests/test_oracle_getrs.py``: LAPACK's getrs (scipy's lu_solve) as a black box,
the residual of P L U X = alpha B, the exact permutation-only case, and the
same interchanges written as a permutation matrix; ``potrs`` against LAPACK's
potrs (scipy's cho_solve) and the residual of L L^H X = alpha B.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "trsm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp", "-std=c99"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (atomic rename)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(prefix="liboracle.", suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def compile_variant(src_text: str, out_dir: str) -> ctypes.CDLL:
    """Compile a modified copy of the oracle source (used by the mutation tests
    that plant a mistake in the oracle to show the pins catch it)."""
    src = os.path.join(out_dir, "oracle_variant.c")
    lib = os.path.join(out_dir, "liboracle_variant.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *CFLAGS, "-o", lib, src, "-lm"], check=True)
    return _bind(ctypes.CDLL(lib))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    i64, dbl, ptr, c_int = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
    lib.oracle_trsm_llnn_d.argtypes = [c_int, i64, i64, dbl, ptr, i64, ptr, i64]
    lib.oracle_trsm_llnn_d.restype = c_int
    lib.oracle_trsm_llnn_z.argtypes = [c_int, i64, i64, ptr, ptr, i64, ptr, i64]
    lib.oracle_trsm_llnn_z.restype = c_int
    lib.oracle_trsm_llnn_cols_d.argtypes = [c_int, i64, dbl, ptr, i64, ptr, i64, ptr, i64]
    lib.oracle_trsm_llnn_cols_d.restype = c_int
    lib.oracle_trsm_llnn_cols_z.argtypes = [c_int, i64, ptr, ptr, i64, ptr, i64, ptr, i64]
    lib.oracle_trsm_llnn_cols_z.restype = c_int
    lib.oracle_trsm_llnn_batch.argtypes = [c_int, c_int, i64, ptr, ptr, ptr, ptr, ptr, ptr, ptr]
    lib.oracle_trsm_llnn_batch.restype = c_int
    lib.oracle_backward_error_d.argtypes = [c_int, i64, i64, dbl, ptr, i64, ptr, i64, ptr, i64]
    lib.oracle_backward_error_d.restype = dbl
    lib.oracle_backward_error_z.argtypes = [c_int, i64, i64, ptr, ptr, i64, ptr, i64, ptr, i64]
    lib.oracle_backward_error_z.restype = dbl
    lib.oracle_trsm_general.argtypes = [c_int, c_int, c_int, c_int, c_int, i64, i64, ptr, ptr, i64, ptr, i64]
    lib.oracle_trsm_general.restype = c_int
    lib.oracle_num_threads.restype = c_int
    lib.oracle_set_num_threads.argtypes = [c_int]
    return lib


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check_fortran(a: np.ndarray, name: str):
    if not a.flags.f_contiguous:
        raise ValueError(f"{name} must be a Fortran-ordered (column-major) array")
    if a.dtype not in (np.float64, np.complex128):
        raise ValueError(f"{name} must be float64 or complex128")


def _alpha_arr(alpha) -> np.ndarray:
    a = complex(alpha)
    return np.array([a.real, a.imag], dtype=np.float64)


def solve(A: np.ndarray, B: np.ndarray, alpha, unit: bool = False, m: int | None = None,
          _lib=None) -> np.ndarray:
    """X = alpha * L^{-1} B (Section 2.1 formula).

    ``A`` is an (lda, >= m) column-major buffer, ``B`` an (ldb, n) one; m
    defaults to ``A.shape[1]``.  Returns a copy of B with rows [0, m) solved;
    padding rows [m, ldb) are copied through unchanged."""
    L = _lib or lib()
    _check_fortran(A, "A")
    _check_fortran(B, "B")
    m = A.shape[1] if m is None else m
    X = np.array(B, order="F", copy=True)
    n = X.shape[1]
    if A.dtype == np.float64:
        rc = L.oracle_trsm_llnn_d(int(unit), m, n, float(np.real(alpha)), _ptr(A), A.shape[0], _ptr(X), X.shape[0])
    else:
        al = _alpha_arr(alpha)
        rc = L.oracle_trsm_llnn_z(int(unit), m, n, _ptr(al), _ptr(A), A.shape[0], _ptr(X), X.shape[0])
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return X


def solve_general(A: np.ndarray, B: np.ndarray, alpha, side: int = 0, uplo: int = 0, trans: int = 0,
                  unit: bool = False, _lib=None) -> np.ndarray:
    """The BLAS triangular-solve variants by definition (the paper's case is side = uplo =
    trans = 0): side 0 solves op(A) X = alpha B (A is m x m), side 1 solves X op(A) = alpha B
    (A is n x n); uplo 0/1 picks the lower/upper triangle of A; trans 0/1/2 is op(A) = A, A^T,
    A^H.  Returns a copy of B with the solution in rows [0, m)."""
    L = _lib or lib()
    _check_fortran(A, "A")
    _check_fortran(B, "B")
    X = np.array(B, order="F", copy=True)
    m, n = (X.shape[0], X.shape[1])
    cx = 1 if np.iscomplexobj(X) else 0
    if np.iscomplexobj(A) != bool(cx) or X.dtype not in (np.float64, np.complex128):
        raise ValueError("A and B must both be float64 or both complex128")
    al = _alpha_arr(alpha)
    rc = L.oracle_trsm_general(cx, side, uplo, trans, int(unit), m, n, _ptr(al), _ptr(A), A.shape[0], _ptr(X),
                               X.shape[0])
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return X


def getrs(LU: np.ndarray, ipiv, B: np.ndarray, alpha, _lib=None) -> np.ndarray:
    """Solve A X = alpha B from A's LU factors as LAPACK getrf packs them (A = P L U: L unit
    lower below the diagonal of LU, U on and above it; ipiv 1-based, row k interchanged with
    row ipiv[k] in order k = 1..m, or None for no interchanges), by the definition
    X = U^{-1} L^{-1} P^T (alpha B): the interchanges applied to B in order, then the two
    triangular solves (Section 1's motivating use of the solve)."""
    Y = np.array(B, order="F", copy=True)
    if ipiv is not None:
        for k, p in enumerate(np.asarray(ipiv, dtype=np.int64)):
            p = int(p) - 1
            if not k <= p < Y.shape[0]:
                raise ValueError("pivot out of range")
            Y[[k, p], :] = Y[[p, k], :]
    Y = solve_general(LU, Y, alpha, 0, 0, 0, True, _lib=_lib)
    return solve_general(LU, Y, 1.0, 0, 1, 0, False, _lib=_lib)


def potrs(Lf: np.ndarray, B: np.ndarray, alpha, _lib=None) -> np.ndarray:
    """Solve A X = alpha B from A's lower Cholesky factor (A = L L^H, L in the lower triangle of
    Lf as LAPACK potrf leaves it), by the definition X = L^{-H} L^{-1} (alpha B): the lower solve,
    then the conjugate-transposed one (transposed for real data)."""
    Y = solve_general(Lf, B, alpha, 0, 0, 0, False, _lib=_lib)
    return solve_general(Lf, Y, 1.0, 0, 0, 2 if np.iscomplexobj(Lf) else 1, False, _lib=_lib)


def solve_cols(A: np.ndarray, B: np.ndarray, alpha, cols, unit: bool = False) -> np.ndarray:
    """Solve only columns ``cols`` of B; returns an (m, len(cols)) array."""
    _check_fortran(A, "A")
    _check_fortran(B, "B")
    L = lib()
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    X = np.array(B, order="F", copy=True)
    m = A.shape[1]
    if A.dtype == np.float64:
        rc = L.oracle_trsm_llnn_cols_d(int(unit), m, float(np.real(alpha)), _ptr(A), A.shape[0],
                                       _ptr(X), X.shape[0], _ptr(cols), len(cols))
    else:
        al = _alpha_arr(alpha)
        rc = L.oracle_trsm_llnn_cols_z(int(unit), m, _ptr(al), _ptr(A), A.shape[0],
                                       _ptr(X), X.shape[0], _ptr(cols), len(cols))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return np.asfortranarray(X[:m, cols])


def solve_batch(As, Bs, alpha, unit: bool = False):
    """Independent solves X_b = alpha L_b^{-1} B_b (lda = ldb = m_b); returns a list."""
    L = lib()
    batch = len(As)
    if batch == 0:
        return []
    is_c = As[0].dtype == np.complex128
    dt = np.complex128 if is_c else np.float64
    ms = np.array([a.shape[0] for a in As], dtype=np.int64)
    ns = np.array([b.shape[1] for b in Bs], dtype=np.int64)
    offA = np.zeros(batch, dtype=np.int64)
    offB = np.zeros(batch, dtype=np.int64)
    offA[1:] = np.cumsum(ms * ms)[:-1]
    offB[1:] = np.cumsum(ms * ns)[:-1]
    Apack = np.concatenate([np.asarray(a, dtype=dt).ravel(order="F") for a in As])
    Bpack = np.concatenate([np.asarray(b, dtype=dt).ravel(order="F") for b in Bs])
    al = _alpha_arr(alpha)
    rc = L.oracle_trsm_llnn_batch(int(is_c), int(unit), batch, _ptr(ms), _ptr(ns), _ptr(al),
                                  _ptr(Apack), _ptr(offA), _ptr(Bpack), _ptr(offB))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    out = []
    for b in range(batch):
        sz = int(ms[b] * ns[b])
        out.append(Bpack[offB[b]:offB[b] + sz].reshape((ms[b], ns[b]), order="F"))
    return out


def backward_error(A: np.ndarray, B: np.ndarray, X: np.ndarray, alpha, unit: bool = False) -> float:
    """||L X - alpha B||_F / (||L||_F ||X||_F + |alpha| ||B||_F), compensated residual."""
    L = lib()
    A = np.asfortranarray(A)
    B = np.asfortranarray(B)
    X = np.asfortranarray(X)
    m, n = A.shape[1], B.shape[1]
    if A.dtype == np.float64:
        return L.oracle_backward_error_d(int(unit), m, n, float(np.real(alpha)), _ptr(A), A.shape[0],
                                         _ptr(B), B.shape[0], _ptr(X), X.shape[0])
    al = _alpha_arr(alpha)
    return L.oracle_backward_error_z(int(unit), m, n, _ptr(al), _ptr(A), A.shape[0],
                                     _ptr(B), B.shape[0], _ptr(X), X.shape[0])


def forward_error(X: np.ndarray, Xref: np.ndarray) -> float:
    """||X - X_ref||_F / ||X_ref||_F (Table 2's normwise relative error)."""
    X = np.asarray(X, dtype=np.complex128 if np.iscomplexobj(Xref) or np.iscomplexobj(X) else np.float64)
    Xref = np.asarray(Xref, dtype=X.dtype)
    den = np.linalg.norm(Xref)
    num = np.linalg.norm(X - Xref)
    return float(num / den) if den > 0 else float(num)


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(t: int) -> None:
    lib().oracle_set_num_threads(int(t))
