"""Writes tests/golden/trsm_integer.txt: small left/lower/no-transpose solves
A X = alpha B (Section 2.1) whose every intermediate is an integer (or a Gaussian
integer) far below 2^53, so the exact solution is representable and any correct
evaluation order reproduces it bit for bit.

A: unit-modulus diagonal (+1 or -1; +i or -i for complex), a sparse strictly lower
part with entries in {-1, 0, 1} (and +-i for complex); B: integers in [-8, 8];
alpha: +1 or -2.  The stored X is computed by the oracle (oracle.solve) and this
script checks it against exact rational forward substitution before writing.

Run: python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

CASES = [  # (dtype, m, n, alpha, density, seed)
    ("r64", 1, 1, 1.0, 0.0, 1),
    ("r64", 17, 5, -2.0, 0.3, 2),
    ("c128", 33, 4, 1.0, 0.15, 3),
    ("r64", 64, 8, 1.0, 0.1, 4),
    ("c128", 100, 3, -2.0, 0.04, 5),
    ("r64", 200, 2, 1.0, 0.02, 6),
]


def make(dtype, m, n, density, seed):
    rng = np.random.default_rng(seed)
    cx = dtype == "c128"
    units = np.array([1, -1, 1j, -1j]) if cx else np.array([1.0, -1.0])
    A = np.zeros((m, m), dtype=np.complex128 if cx else np.float64)
    A[np.diag_indices(m)] = rng.choice(units, m)
    low = np.tril(rng.random((m, m)) < density, -1)
    A[low] = rng.choice(units, int(low.sum()))
    B = rng.integers(-8, 9, (m, n)).astype(A.dtype)
    if cx:
        B = B + 1j * rng.integers(-8, 9, (m, n))
    return np.asfortranarray(A), np.asfortranarray(B)


def exact_solve(A, B, alpha):
    """Forward substitution in exact Gaussian-rational arithmetic (pairs of Fractions)."""
    m, n = B.shape

    def fr(z):
        z = complex(z)
        return (Fraction(z.real), Fraction(z.imag))

    def mul(a, b):
        return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])

    def div(a, b):
        d = b[0] * b[0] + b[1] * b[1]
        return ((a[0] * b[0] + a[1] * b[1]) / d, (a[1] * b[0] - a[0] * b[1]) / d)

    al = fr(alpha)
    X = [[None] * n for _ in range(m)]
    for j in range(n):
        for i in range(m):
            s = mul(al, fr(B[i, j]))
            for k in range(i):
                if A[i, k] != 0:
                    p = mul(fr(A[i, k]), X[k][j])
                    s = (s[0] - p[0], s[1] - p[1])
            X[i][j] = div(s, fr(A[i, i]))
    return X


def main():
    lines = ["# Integer-valued left/lower/no-transpose solves A X = alpha B (Section 2.1).",
             "# Written by tests/golden/make_golden.py: X from oracle.solve, checked exactly.",
             "# Per case: 'case dtype m n alpha'; then 'A i k re im' for each nonzero of the",
             "# lower triangle; then 'B i j re im' and 'X i j re im' for every entry."]
    for dtype, m, n, alpha, density, seed in CASES:
        A, B = make(dtype, m, n, density, seed)
        X = oracle.solve(A, B, alpha)
        Xe = exact_solve(A, B, alpha)
        for i in range(m):
            for j in range(n):
                re, im = Xe[i][j]
                assert re.denominator == 1 and im.denominator == 1 and abs(re) < 2 ** 50 and abs(im) < 2 ** 50
                assert complex(X[i, j]) == complex(float(re), float(im)), (dtype, m, i, j)
        lines.append(f"case {dtype} {m} {n} {alpha!r}")
        for i, k in zip(*np.nonzero(np.tril(A))):
            z = complex(A[i, k])
            lines.append(f"A {i} {k} {z.real:.0f} {z.imag:.0f}")
        for name, M in (("B", B), ("X", X)):
            for j in range(n):
                for i in range(m):
                    z = complex(M[i, j])
                    lines.append(f"{name} {i} {j} {z.real:.0f} {z.imag:.0f}")
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "trsm_integer.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
