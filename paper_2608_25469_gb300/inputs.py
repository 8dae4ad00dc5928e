"""Seeded synthetic inputs for the triangular solve (host side).

This module is the only code shared by the CUDA path's tests/benchmarks and the
oracle's tests.  It holds none of the solve's arithmetic: it only draws numbers.

Generator
---------
A counter-based SplitMix64 (S. Vigna, public domain; the finaliser is the one of
Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
2014).  Output ``i`` of stream ``s`` under ``seed`` is the ``i``-th output of a
SplitMix64 sequence whose state starts at ``key(seed, s)``::

    mix64(z)  = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)
    key(seed, s) = mix64(seed * G + s * H + G)            (mod 2^64)
    u64(seed, s, i) = mix64(key(seed, s) + (i + 1) * G)   (mod 2^64)
    u01 = (u64 >> 11) * 2^-53                              in [0, 1)

with G = 0x9E3779B97F4A7C15 and H = 0xD1B54A32D192ED03.  The device side
(``csrc/gen.cu``) implements the same definition; tests check the two agree
bit for bit.

Streams (the low 8 bits) and the instance id (the bits above) address the
draws: ``stream = base + ((inst + 1) << 8)``, ``inst = -1`` for a single solve.

Workload recipe (the configurations the paper's evaluation uses, Section 5.1:
random square matrices; the distributions below are this library's reading)
----------------------------------------------------------------------------
* A (m x m, column-major, element index i + j*m): A_ij = (2u - 1)/m for i > j,
  A_ii = 1 + u, A_ij = 0 for i < j.  Complex: real and imaginary parts drawn
  independently in the same way (streams A_RE and A_IM).
* B (m x n, column-major, index i + j*m): B_ij = 2u - 1 (streams B_RE, B_IM).
* Packed LU factors (kind 2): below the diagonal A's multipliers; on and above
  it the transpose of a second triangle drawn like A from streams U_RE, U_IM.
* Batched small sizes: m, n uniform on {8, ..., 64}.
* Serving stream: m = floor(exp(U(ln 16, ln 4097))) clamped to [16, 4096],
  n = floor(exp(U(0, ln 513))) clamped to [1, 512], fp64 with probability 0.7
  (else complex128), exponential inter-arrival gaps at a given rate.
"""
from __future__ import annotations

import numpy as np

G = 0x9E3779B97F4A7C15
H = 0xD1B54A32D192ED03
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1

A_RE, B_RE, A_IM, B_IM = 0, 1, 2, 3
U_RE, U_IM = 4, 5  # the upper factor of generated packed LU factors
SIZE_M, SIZE_N, DTYPE_SEL, ARRIVAL = 16, 17, 18, 19

R64, C128 = 0, 1  # dtype codes, identical to the C-ABI's


def _mix64_int(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def stream_id(base: int, inst: int = -1) -> int:
    """Stream number for draw family ``base`` of instance ``inst``."""
    return (base + ((inst + 1) << 8)) & MASK


def key(seed: int, stream: int) -> int:
    return _mix64_int((seed * G + stream * H + G) & MASK)


def _mix64_arr(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(M1)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(M2)
    return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, idx) -> np.ndarray:
    """Raw 64-bit draws ``u64(seed, stream, i)`` for every i in ``idx``."""
    idx = np.asarray(idx, dtype=np.uint64)
    k = np.uint64(key(seed, stream))
    with np.errstate(over="ignore"):
        z = k + (idx + np.uint64(1)) * np.uint64(G)
        return _mix64_arr(z)


def u01(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform draws in [0, 1) with 53 random bits."""
    return (u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _tri_from_uniform(m: int, ua: np.ndarray) -> np.ndarray:
    """Lower-triangular m x m (column-major index) from uniforms: the recipe above."""
    ua = ua.reshape((m, m), order="F")
    i = np.arange(m)[:, None]
    j = np.arange(m)[None, :]
    off = (2.0 * ua - 1.0) / m
    diag = 1.0 + ua
    return np.where(i > j, off, np.where(i == j, diag, 0.0))


def gen_A(seed: int, m: int, dtype: int = R64, inst: int = -1) -> np.ndarray:
    """A for one solve, shape (m, m), Fortran order; float64 or complex128."""
    idx = np.arange(m * m, dtype=np.uint64)
    re = _tri_from_uniform(m, u01(seed, stream_id(A_RE, inst), idx))
    if dtype == R64:
        return np.asfortranarray(re)
    im = _tri_from_uniform(m, u01(seed, stream_id(A_IM, inst), idx))
    return np.asfortranarray(re + 1j * im)


def gen_LU(seed: int, m: int, dtype: int = R64, inst: int = -1) -> np.ndarray:
    """Packed LU factors (LAPACK getrf layout, no interchanges), shape (m, m), Fortran
    order: below the diagonal the multipliers of gen_A's lower triangle (streams A_RE,
    A_IM); on and above it U = T^T, T drawn as gen_A draws A but from streams U_RE, U_IM
    (so U_ii = 1 + u and U_ij = (2u - 1)/m, element (i, j) of U taking T's index j + i m)."""
    idx = np.arange(m * m, dtype=np.uint64)
    parts = []
    for sa, su in ((A_RE, U_RE), (A_IM, U_IM))[:1 if dtype == R64 else 2]:
        L = _tri_from_uniform(m, u01(seed, stream_id(sa, inst), idx))
        T = _tri_from_uniform(m, u01(seed, stream_id(su, inst), idx))
        parts.append(np.tril(L, -1) + T.T)
    if dtype == R64:
        return np.asfortranarray(parts[0])
    return np.asfortranarray(parts[0] + 1j * parts[1])


def gen_B(seed: int, m: int, n: int, dtype: int = R64, inst: int = -1) -> np.ndarray:
    """B for one solve, shape (m, n), Fortran order; float64 or complex128."""
    idx = np.arange(m * n, dtype=np.uint64)
    re = (2.0 * u01(seed, stream_id(B_RE, inst), idx) - 1.0).reshape((m, n), order="F")
    if dtype == R64:
        return np.asfortranarray(re)
    im = (2.0 * u01(seed, stream_id(B_IM, inst), idx) - 1.0).reshape((m, n), order="F")
    return np.asfortranarray(re + 1j * im)


def gen_B_cols(seed: int, m: int, cols, dtype: int = R64, inst: int = -1) -> np.ndarray:
    """Selected columns of B (the same values gen_B would give), shape (m, len(cols))."""
    cols = np.asarray(cols, dtype=np.uint64)
    idx = (np.arange(m, dtype=np.uint64)[:, None] + cols[None, :] * np.uint64(m)).ravel(order="F")
    shape = (m, len(cols))
    re = (2.0 * u01(seed, stream_id(B_RE, inst), idx) - 1.0).reshape(shape, order="F")
    if dtype == R64:
        return np.asfortranarray(re)
    im = (2.0 * u01(seed, stream_id(B_IM, inst), idx) - 1.0).reshape(shape, order="F")
    return np.asfortranarray(re + 1j * im)


def batched_sizes(seed: int, batch: int, lo: int = 8, hi: int = 64):
    """(m_i, n_i) for the varlen batched workload: each uniform on {lo, ..., hi}."""
    idx = np.arange(batch, dtype=np.uint64)
    span = hi - lo + 1
    m = lo + np.floor(u01(seed, SIZE_M, idx) * span).astype(np.int64)
    n = lo + np.floor(u01(seed, SIZE_N, idx) * span).astype(np.int64)
    return np.minimum(m, hi), np.minimum(n, hi)


def serving_requests(seed: int, count: int, rate_per_s: float = 2000.0,
                     m_range=(16, 4096), n_range=(1, 512), p_fp64: float = 0.7):
    """Request stream: arrival times (s), m, n, dtype code per request."""
    idx = np.arange(count, dtype=np.uint64)
    um = u01(seed, SIZE_M, idx)
    un = u01(seed, SIZE_N, idx)
    ud = u01(seed, DTYPE_SEL, idx)
    ua = u01(seed, ARRIVAL, idx)
    m = np.floor(np.exp(np.log(m_range[0]) + um * (np.log(m_range[1] + 1) - np.log(m_range[0]))))
    n = np.floor(np.exp(np.log(n_range[0]) + un * (np.log(n_range[1] + 1) - np.log(n_range[0]))))
    m = np.clip(m, m_range[0], m_range[1]).astype(np.int64)
    n = np.clip(n, n_range[0], n_range[1]).astype(np.int64)
    dt = np.where(ud < p_fp64, R64, C128).astype(np.int64)
    gaps = -np.log1p(-ua) / rate_per_s
    return np.cumsum(gaps), m, n, dt


def embed(X: np.ndarray, ld: int, fill=np.nan) -> np.ndarray:
    """Copy X (rows x cols) into a column-major buffer with leading dimension ``ld``.

    Returns the (ld, cols) Fortran-ordered buffer; rows >= X.shape[0] hold ``fill``
    (canaries for padding checks)."""
    rows, cols = X.shape
    out = np.full((ld, cols), fill, dtype=X.dtype, order="F")
    out[:rows, :] = X
    return out


def flops_trsm(m, n, complex_: bool) -> float:
    """Counted flops of one solve: m^2 n real, x4 for complex."""
    f = float(m) * float(m) * float(n)
    return 4.0 * f if complex_ else f


__all__ = [
    "u64", "u01", "key", "stream_id", "gen_A", "gen_B", "gen_B_cols", "batched_sizes",
    "serving_requests", "embed", "flops_trsm", "R64", "C128", "gen_LU",
    "A_RE", "B_RE", "A_IM", "B_IM", "U_RE", "U_IM",
]
