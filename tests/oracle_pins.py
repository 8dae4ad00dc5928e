"""Pins for the oracle: checks against facts fixed by mathematics, not by the oracle.

Each ``pin_*`` function takes a ``solve(A, B, alpha, unit)`` callable (the
oracle, or a deliberately broken copy of it in the mutation tests) and raises
AssertionError when the callable disagrees with the fact it pins.

The facts (all about L X = alpha B, L lower triangular; Section 2.1):
* identity A: X = alpha B;
* diagonal A: X = alpha B / diag (one rounding per operation);
* unit lower bidiagonal A with sub-diagonal c: x_i = alpha sum_{k<=i} (-c)^{i-k} b_k,
  exact in binary floating point for integer data and c in {-1, +1, 1/2, i};
* exact rational Gaussian elimination on small dyadic inputs (Python
  ``fractions``), with Higham's componentwise forward-error bound for
  substitution (Accuracy and Stability of Numerical Algorithms, 2nd ed., Thm 8.5);
* LAPACK's triangular solve via ``scipy.linalg.solve_triangular`` (a library
  called as a black box);
* invariants: the strict upper triangle and (with a unit diagonal) the diagonal
  are never read; columns are independent; complex data with zero imaginary
  parts reproduces the real solve; padding rows are untouched; scaling alpha by
  a power of two scales X exactly.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

U = 2.0 ** -53


def _rng(seed):
    return np.random.default_rng(seed)


def _F(x):
    return np.asfortranarray(x)


def pin_identity(solve, dtype=np.float64):
    rng = _rng(1)
    m, n = 17, 5
    A = _F(np.eye(m, dtype=dtype))
    B = rng.uniform(-1, 1, (m, n))
    alpha = 1.75
    if dtype == np.complex128:
        B = B + 1j * rng.uniform(-1, 1, (m, n))
        alpha = 1.5 - 0.5j
    B = _F(B.astype(dtype))
    X = solve(A, B, alpha, False)
    if dtype == np.float64:
        assert np.array_equal(X, alpha * B), "identity: X != alpha B"
    else:
        # one complex product per element: each part within 2 ulp of the exact value
        exact_re = np.array([[float(Fraction(alpha.real) * Fraction(b.real) - Fraction(alpha.imag) * Fraction(b.imag))
                              for b in row] for row in B])
        exact_im = np.array([[float(Fraction(alpha.real) * Fraction(b.imag) + Fraction(alpha.imag) * Fraction(b.real))
                              for b in row] for row in B])
        scale = np.abs(alpha) * np.abs(B)
        assert np.all(np.abs(X.real - exact_re) <= 4 * U * scale), "identity (complex): real part"
        assert np.all(np.abs(X.imag - exact_im) <= 4 * U * scale), "identity (complex): imaginary part"


def pin_diagonal(solve, dtype=np.float64):
    rng = _rng(2)
    m, n = 23, 4
    d = rng.uniform(0.5, 3.0, m)
    B = rng.uniform(-1, 1, (m, n))
    alpha = -1.25
    if dtype == np.complex128:
        d = d + 1j * rng.uniform(-2.0, 2.0, m)
        B = B + 1j * rng.uniform(-1, 1, (m, n))
        alpha = 0.75 + 1.0j
    A = _F(np.diag(d).astype(dtype))
    B = _F(B.astype(dtype))
    X = solve(A, B, alpha, False)
    if dtype == np.float64:
        assert np.array_equal(X, (alpha * B) / d[:, None]), "diagonal: X != (alpha B) / d"
    else:
        exact = (alpha * B) / d[:, None]
        assert np.all(np.abs(X - exact) <= 16 * U * np.abs(exact)), "diagonal (complex)"


def bidiagonal_closed_form(b_col, alpha, c):
    """x_i = alpha * sum_{k<=i} (-c)^{i-k} b_k, exactly (Fractions / Gaussian rationals)."""
    out = []
    acc_re, acc_im = Fraction(0), Fraction(0)
    cre, cim = Fraction(c.real), Fraction(c.imag)
    for bk in b_col:
        # acc <- alpha*b_k - c*acc
        are, aim = Fraction(alpha.real), Fraction(alpha.imag)
        bre, bim = Fraction(bk.real), Fraction(bk.imag)
        t_re = are * bre - aim * bim - (cre * acc_re - cim * acc_im)
        t_im = are * bim + aim * bre - (cre * acc_im + cim * acc_re)
        acc_re, acc_im = t_re, t_im
        out.append(complex(float(acc_re), float(acc_im)))
    return np.array(out)


def pin_bidiagonal(solve, dtype=np.float64):
    rng = _rng(3)
    cases = [(-1.0, 60, 1.0), (1.0, 60, 2.0), (0.5, 40, 1.0)]
    if dtype == np.complex128:
        cases += [(1j, 50, 1.0 + 0j), (-1.0, 50, 1.0 - 1.0j)]
    for c, m, alpha in cases:
        n = 3
        B = rng.integers(-8, 9, (m, n)).astype(np.float64)
        if dtype == np.complex128:
            B = B + 1j * rng.integers(-8, 9, (m, n))
        B = _F(B.astype(dtype))
        A = np.eye(m, dtype=dtype) + np.diag(np.full(m - 1, c, dtype=dtype), -1)
        for unit in (False, True):
            Au = A.copy()
            if unit:
                np.fill_diagonal(Au, np.nan)  # never read under a unit diagonal
            X = solve(_F(Au), B, alpha, unit)
            for j in range(n):
                ref = bidiagonal_closed_form(B[:, j].astype(np.complex128), complex(alpha), complex(c))
                got = X[:, j].astype(np.complex128)
                assert np.array_equal(got, ref), f"bidiagonal c={c} unit={unit}: mismatch in column {j}"


def _exact_solve(L, b, alpha):
    """Exact forward substitution over Q (or Q[i]) for small inputs; L given as nested lists of Fractions pairs."""
    m = len(b)
    x = []
    for i in range(m):
        sr = alpha[0] * b[i][0] - alpha[1] * b[i][1]
        si = alpha[0] * b[i][1] + alpha[1] * b[i][0]
        for k in range(i):
            ar, ai = L[i][k]
            sr -= ar * x[k][0] - ai * x[k][1]
            si -= ar * x[k][1] + ai * x[k][0]
        dr, di = L[i][i]
        den = dr * dr + di * di
        x.append(((sr * dr + si * di) / den, (si * dr - sr * di) / den))
    return x


def pin_exact_rational(solve, dtype=np.float64):
    """Brute force over Q on 4x4 to 8x8 dyadic inputs, with Higham's bound."""
    rng = _rng(4)
    cplx = dtype == np.complex128
    for m in (4, 5, 8):
        n = 3
        Ar = rng.integers(-16, 17, (m, m)) / 8.0
        Ai = rng.integers(-16, 17, (m, m)) / 8.0 if cplx else np.zeros((m, m))
        dr = rng.choice([1.0, 1.5, 3.0, 5.0, 7.0, 0.75], m)
        di = rng.choice([0.0, 0.5, -1.25], m) if cplx else np.zeros(m)
        Ar = np.tril(Ar, -1) + np.diag(dr)
        Ai = np.tril(Ai, -1) + np.diag(di)
        Br = rng.integers(-16, 17, (m, n)) / 4.0
        Bi = rng.integers(-16, 17, (m, n)) / 4.0 if cplx else np.zeros((m, n))
        alpha = complex(1.5, -0.5) if cplx else complex(1.5, 0.0)
        A = Ar + 1j * Ai if cplx else Ar
        B = Br + 1j * Bi if cplx else Br
        A = _F(A.astype(dtype))
        B = _F(B.astype(dtype))
        X = solve(A, B, alpha if cplx else alpha.real, False)
        Lq = [[(Fraction(Ar[i, k]), Fraction(Ai[i, k])) for k in range(m)] for i in range(m)]
        al = (Fraction(alpha.real), Fraction(alpha.imag))
        Labs = np.abs(A)
        Linv_abs = np.abs(np.linalg.inv(A.astype(np.complex128)))
        gamma = (6 * m + 12) * U / (1 - (6 * m + 12) * U)
        for j in range(n):
            bq = [(Fraction(Br[i, j]), Fraction(Bi[i, j])) for i in range(m)]
            xq = _exact_solve(Lq, bq, al)
            xe = np.array([complex(float(a), float(b)) for a, b in xq])
            bound = gamma * (Linv_abs @ (Labs @ np.abs(xe)) + Linv_abs @ (abs(alpha) * np.abs(B[:, j])))
            err = np.abs(X[:, j].astype(np.complex128) - xe)
            assert np.all(err <= bound + 1e-300), f"exact rational m={m} col {j}: err {err.max()} > bound"


def pin_lapack(solve, dtype=np.float64):
    import scipy.linalg as sl
    rng = _rng(5)
    for m, n, pad in ((1, 1, 0), (5, 3, 2), (64, 64, 0), (100, 7, 3), (257, 11, 1)):
        A = np.tril(rng.uniform(-1, 1, (m, m)) / m, -1) + np.diag(1 + rng.uniform(0, 1, m))
        B = rng.uniform(-1, 1, (m, n))
        alpha = 1.5
        if dtype == np.complex128:
            A = A + 1j * (np.tril(rng.uniform(-1, 1, (m, m)) / m, -1) + np.diag(1 + rng.uniform(0, 1, m)))
            B = B + 1j * rng.uniform(-1, 1, (m, n))
            alpha = 1.5 - 0.5j
        Ab = np.full((m + pad, m), np.nan, dtype=dtype, order="F")
        Ab[:m] = np.tril(A)
        Ab[:m][np.triu_indices(m, 1)] = np.nan  # strict upper triangle is never read
        Bb = np.full((m + pad, n), 7.0, dtype=dtype, order="F")
        Bb[:m] = B
        X = solve(Ab, Bb, alpha, False)
        ref = sl.solve_triangular(np.tril(A), alpha * B, lower=True)
        err = np.linalg.norm(X[:m] - ref) / np.linalg.norm(ref)
        assert err <= 1e-14, f"LAPACK cross-check m={m} n={n}: {err}"
        assert np.all(X[m:] == 7.0), "padding rows changed"


def pin_invariants(solve, dtype=np.float64):
    rng = _rng(6)
    m, n = 33, 9
    A = np.tril(rng.uniform(-1, 1, (m, m)) / m, -1) + np.diag(1 + rng.uniform(0, 1, m))
    B = rng.uniform(-1, 1, (m, n))
    alpha = 0.75
    if dtype == np.complex128:
        A = A + 1j * np.tril(rng.uniform(-1, 1, (m, m)), 0) / m
        B = B + 1j * rng.uniform(-1, 1, (m, n))
        alpha = 0.75 + 0.25j
    A = _F(A.astype(dtype))
    B = _F(B.astype(dtype))
    X = solve(A, B, alpha, False)
    # upper triangle never read
    Ap = A.copy()
    Ap[np.triu_indices(m, 1)] = np.nan
    assert np.array_equal(solve(_F(Ap), B, alpha, False), X), "upper triangle was read"
    # unit diagonal never read; equals a solve with an explicit unit diagonal
    Au = A.copy()
    np.fill_diagonal(Au, np.nan)
    A1 = A.copy()
    np.fill_diagonal(A1, 1.0)
    assert np.array_equal(solve(_F(Au), B, alpha, True), solve(_F(A1), B, alpha, False)), "unit diagonal"
    # columns independent
    for j in (0, 4, n - 1):
        Xj = solve(A, _F(B[:, j:j + 1]), alpha, False)
        assert np.array_equal(Xj[:, 0], X[:, j]), "column solved alone differs"
    # power-of-two alpha scaling is exact
    assert np.array_equal(solve(A, B, 2 * alpha, False), 2 * X), "alpha scaling"
    # alpha = 0: B := 0 without reading A
    Anan = _F(np.full((m, m), np.nan, dtype=dtype))
    assert np.array_equal(solve(Anan, B, 0.0, False), np.zeros_like(B)), "alpha = 0"
    if dtype == np.complex128:
        # zero imaginary parts reproduce the real solve
        Ar = _F(A.real.copy())
        Br = _F(B.real.copy())
        Xr = solve(Ar, Br, alpha.real, False)
        Xc = solve(_F(Ar.astype(np.complex128)), _F(Br.astype(np.complex128)), complex(alpha.real, 0.0), False)
        assert np.array_equal(Xc.real, Xr) and np.all(Xc.imag == 0), "complex with zero imaginary part"


ALL_PINS = [pin_identity, pin_diagonal, pin_bidiagonal, pin_exact_rational, pin_lapack, pin_invariants]
