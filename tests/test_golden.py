"""The integer-valued golden solves (tests/golden/trsm_integer.txt, written by
tests/golden/make_golden.py from the oracle): the stored X satisfies A X = alpha B
exactly in integer arithmetic (a check by multiplication, independent of how X was
computed; X is unique since A is triangular with a nonzero diagonal), and the oracle
reproduces it bit for bit."""
import numpy as np

import oracle
from tests import golden_cases


def _exact_residual_zero(A, B, alpha, X):
    m, n = B.shape
    for j in range(n):
        for i in range(m):
            s = 0
            for k in range(i + 1):
                if A[i, k] != 0:
                    a, x = complex(A[i, k]), complex(X[k, j])
                    s += complex(int(a.real), int(a.imag)) * complex(int(x.real), int(x.imag))
            b = complex(B[i, j]) * alpha
            if s != b:
                return False
    return True


def test_golden_cases_cover_small_and_blocked_sizes():
    ms = sorted(A.shape[0] for _, A, _, _, _ in golden_cases.load())
    assert ms[0] == 1 and ms[-1] > 64 and any(m == 64 for m in ms)
    assert {d for d, *_ in golden_cases.load()} == {"r64", "c128"}


def test_golden_x_solves_exactly():
    for dtype, A, B, alpha, X in golden_cases.load():
        assert np.all(X == np.round(X.real) + 1j * np.round(X.imag) if dtype == "c128" else X == np.round(X))
        assert np.max(np.abs(X)) < 2 ** 40
        assert _exact_residual_zero(A, B, alpha, X), (dtype, A.shape)


def test_oracle_reproduces_golden_bitwise():
    for dtype, A, B, alpha, X in golden_cases.load():
        assert np.array_equal(oracle.solve(A, B, alpha), X), (dtype, A.shape)
