"""Pins for the oracle's BLAS variants (side, uplo, trans, diag), by means other
than the oracle itself: the left/lower/no-transpose case equals the pinned
forward-substitution oracle bit for bit; LAPACK (scipy.linalg.solve_triangular,
as a black box) agrees for every variant; a diagonal A gives alpha B / d
exactly; the residual op(A) X - alpha B (or X op(A) - alpha B) is at rounding
level; the untouched triangle and a unit diagonal are never read.  Planted
mistakes in a compiled copy of the oracle are caught."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I

VARIANTS = list(itertools.product((0, 1), (0, 1), (0, 1, 2), (False, True)))  # side, uplo, trans, unit


def _problem(seed, side, uplo, cx, m=37, n=23):
    code = I.C128 if cx else I.R64
    na = m if side == 0 else n
    L = I.gen_A(seed, na, code)
    A = np.asfortranarray(L if uplo == 0 else L.T.copy())  # lower, or its transpose (upper)
    B = I.gen_B(seed + 1, m, n, code)
    return A, B


def _op(A, trans, uplo, unit):
    T = np.tril(A) if uplo == 0 else np.triu(A)
    if unit:
        T = T - np.diag(np.diag(T)) + np.eye(T.shape[0])
    return T if trans == 0 else (T.T if trans == 1 else T.conj().T)


def _scipy_ref(A, B, alpha, side, uplo, trans, unit):
    la = pytest.importorskip("scipy.linalg")
    rhs = alpha * B
    if side == 0:
        return la.solve_triangular(A, rhs, lower=(uplo == 0), trans=trans, unit_diagonal=unit)
    # X op(A) = rhs  <=>  op(A)^T X^T = rhs^T
    if trans == 0:
        Y = la.solve_triangular(A, rhs.T, lower=(uplo == 0), trans=1, unit_diagonal=unit)
    elif trans == 1:
        Y = la.solve_triangular(A, rhs.T, lower=(uplo == 0), trans=0, unit_diagonal=unit)
    else:  # op(A)^T = conj(A)
        Y = la.solve_triangular(A.conj(), rhs.T, lower=(uplo == 0), trans=0, unit_diagonal=unit)
    return Y.T


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("unit", [False, True])
def test_left_lower_notrans_equals_pinned_oracle(cx, unit):
    A, B = _problem(3, 0, 0, cx)
    alpha = 1.5 - 0.5j if cx else 1.5
    assert np.array_equal(oracle.solve_general(A, B, alpha, 0, 0, 0, unit), oracle.solve(A, B, alpha, unit))


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("side,uplo,trans,unit", VARIANTS)
def test_variants_match_lapack_and_residual(cx, side, uplo, trans, unit):
    A, B = _problem(11 + 3 * side + uplo, side, uplo, cx)
    alpha = 0.75 + 1.25j if cx else -1.25
    X = oracle.solve_general(A, B, alpha, side, uplo, trans, unit)
    assert _rel(X, _scipy_ref(A, B, alpha, side, uplo, trans, unit)) <= 1e-13
    T = _op(A, trans, uplo, unit)
    R = (T @ X if side == 0 else X @ T) - alpha * B
    scale = (np.abs(T) @ np.abs(X) if side == 0 else np.abs(X) @ np.abs(T)) + abs(alpha) * np.abs(B)
    assert np.max(np.abs(R) / scale) <= 64 * np.finfo(np.float64).eps


@pytest.mark.parametrize("side,uplo,trans,unit", VARIANTS)
def test_diagonal_closed_form(side, uplo, trans, unit):
    m, n = 9, 6
    na = m if side == 0 else n
    d = 1.0 + np.arange(na) / 8.0
    A = np.asfortranarray(np.diag(d))
    B = np.asfortranarray(np.arange(m * n, dtype=np.float64).reshape(m, n, order="F") - 20.0)
    X = oracle.solve_general(A, B, 1.5, side, uplo, trans, unit)
    if unit:
        assert np.array_equal(X, 1.5 * B)
    else:
        assert np.array_equal(X, (1.5 * B) / (d[:, None] if side == 0 else d[None, :]))


@pytest.mark.parametrize("side,uplo,trans", [v[:3] for v in VARIANTS if not v[3]])
def test_unreferenced_triangle_and_unit_diagonal_not_read(side, uplo, trans):
    A, B = _problem(5, side, uplo, True)
    ref = oracle.solve_general(A, B, 2.0, side, uplo, trans, False)
    P = A.copy(order="F")
    na = P.shape[0]
    other = np.tril_indices(na, -1) if uplo == 1 else np.triu_indices(na, 1)
    P[other] = np.nan
    assert np.array_equal(oracle.solve_general(P, B, 2.0, side, uplo, trans, False), ref)
    refu = oracle.solve_general(A, B, 2.0, side, uplo, trans, True)
    P[np.diag_indices(na)] = np.nan
    assert np.array_equal(oracle.solve_general(P, B, 2.0, side, uplo, trans, True), refu)


MUTANTS = {
    "transpose ignored in the substitution order": ("const int t_lower = (uplo == 0) != (trans != 0);",
                                                    "const int t_lower = (uplo == 0);"),
    "conjugation dropped": ("if (trans == 2) v.im = -v.im;", "(void)0;"),
    "right side multiplies on the wrong side": (
        "s = z_sub(s, z_mul(g_get(cx, B, ldb, i, l), g_op(cx, trans, A, lda, l, k)));",
        "s = z_sub(s, z_mul(g_get(cx, B, ldb, i, l), g_op(cx, trans, A, lda, k, l)));"),
    "backward substitution skips a term": ("const int64_t k0 = t_lower ? 0 : i + 1, k1 = t_lower ? i : m;",
                                           "const int64_t k0 = t_lower ? 0 : i + 2, k1 = t_lower ? i : m;"),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_general_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation site for '{name}' not found"
    lib = oracle.compile_variant(src.replace(old, new, 1), str(tmp_path))
    caught = False
    for cx in (False, True):
        for side, uplo, trans, unit in VARIANTS:
            A, B = _problem(11 + 3 * side + uplo, side, uplo, cx)
            alpha = 0.75 + 1.25j if cx else -1.25
            X = oracle.solve_general(A, B, alpha, side, uplo, trans, unit, _lib=lib)
            if not _rel(X, _scipy_ref(A, B, alpha, side, uplo, trans, unit)) <= 1e-13:
                caught = True
                break
        if caught:
            break
    assert caught, f"no pin caught the planted mistake '{name}'"
