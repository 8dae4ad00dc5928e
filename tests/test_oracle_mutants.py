"""Plant plausible mistakes in a copy of the oracle's source and show the pins catch each.

The mistakes are planted in a temporary copy compiled on the CPU; the oracle
itself is never modified.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests import oracle_pins as P

MUTANTS = {
    "transposed operand": ("const double *ak = A + k * lda;\n    for (int64_t i = k + 1; i < m; i++) x[i] = x[i] - ak[i] * xk;",
                           "for (int64_t i = k + 1; i < m; i++) x[i] = x[i] - A[k + i * lda] * xk;"),
    "dropped diagonal division": ("if (!unit) x[k] = x[k] / A[k + k * lda];", "(void)0;"),
    "sign of update": ("x[i] = x[i] - ak[i] * xk;", "x[i] = x[i] + ak[i] * xk;"),
    "dropped alpha": ("for (int64_t i = 0; i < m; i++) x[i] = alpha * x[i];", "(void)alpha;"),
    "skipped first sub-diagonal term": ("for (int64_t i = k + 1; i < m; i++) x[i] = x[i] - ak[i] * xk;",
                                        "for (int64_t i = k + 2; i < m; i++) x[i] = x[i] - ak[i] * xk;"),
    "complex product sign": ("r.im = a.re * b.im + a.im * b.re;", "r.im = a.re * b.im - a.im * b.re;"),
    "complex division conjugated": ("r.im = (a.im - a.re * t) / d;", "r.im = (a.re * t - a.im) / d;"),
    "complex update uses diagonal index": ("x[i] = z_sub(x[i], z_mul(ak[i], xk));",
                                           "x[i] = z_sub(x[i], z_mul(ak[k], xk));"),
}


def _solver(lib):
    def solve(A, B, alpha, unit):
        return oracle.solve(A, B, alpha, unit, _lib=lib)
    return solve


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) >= 1, f"mutation site for '{name}' not found"
    lib = oracle.compile_variant(src.replace(old, new, 1), str(tmp_path))
    solve = _solver(lib)
    caught = []
    for dtype in (np.float64, np.complex128):
        for pin in P.ALL_PINS:
            try:
                pin(solve, dtype)
            except (AssertionError, ValueError, FloatingPointError):
                caught.append((pin.__name__, dtype.__name__))
    assert caught, f"no pin caught the planted mistake '{name}'"


def test_unmodified_copy_passes_all_pins(tmp_path):
    lib = oracle.compile_variant(oracle.source_text(), str(tmp_path))
    solve = _solver(lib)
    for dtype in (np.float64, np.complex128):
        for pin in P.ALL_PINS:
            pin(solve, dtype)
