"""The oracle against facts fixed by mathematics (CPU only)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import oracle_pins as P

DTYPES = [np.float64, np.complex128]


def _solve(A, B, alpha, unit):
    return oracle.solve(A, B, alpha, unit)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin, dtype):
    pin(_solve, dtype)


@pytest.mark.parametrize("dtype", [I.R64, I.C128])
@pytest.mark.parametrize("m,n", [(64, 64), (1, 1), (8, 64), (64, 8), (300, 17)])
def test_backward_error_seeded(dtype, m, n):
    """Normwise backward error of the oracle on the seeded workload generator <= 1e-14."""
    A = I.gen_A(0, m, dtype)
    B = I.gen_B(0, m, n, dtype)
    alpha = 1.5 if dtype == I.R64 else 1.5 - 0.5j
    X = oracle.solve(A, B, alpha)
    eta = oracle.backward_error(A, B, X, alpha)
    assert eta <= 1e-14, eta


def test_backward_error_checker_exact_solution_is_zero():
    """The checker returns exactly 0 for an exact solution (prefix-sum case)."""
    m, n = 40, 3
    rng = np.random.default_rng(7)
    B = np.asfortranarray(rng.integers(-8, 9, (m, n)).astype(np.float64))
    A = np.asfortranarray(np.eye(m) - np.diag(np.ones(m - 1), -1))
    X = np.asfortranarray(np.cumsum(B, axis=0))
    assert oracle.backward_error(A, B, X, 1.0) == 0.0
    Bz = np.asfortranarray(B + 1j * B[::-1])
    Xz = np.asfortranarray(np.cumsum(Bz, axis=0))
    assert oracle.backward_error(np.asfortranarray(A.astype(complex)), Bz, Xz, 1.0 + 0j) == 0.0


@pytest.mark.parametrize("cplx", [False, True])
def test_backward_error_checker_known_residual(cplx):
    """Perturb one entry of an exact solution: the residual is L delta e_ij, known exactly."""
    m, n = 6, 2
    rng = np.random.default_rng(8)
    L = np.tril(rng.integers(-4, 5, (m, m)) / 4.0, -1) + np.diag(rng.choice([1.0, 2.0, 4.0], m))
    if cplx:
        L = L + 1j * np.tril(rng.integers(-4, 5, (m, m)) / 4.0, -1)
    X = rng.integers(-4, 5, (m, n)).astype(np.float64) + (1j * rng.integers(-4, 5, (m, n)) if cplx else 0)
    B = L @ X  # exact: small dyadic integers
    delta = 2.0 ** -20
    Xp = X.copy()
    Xp[2, 1] += delta
    eta = oracle.backward_error(np.asfortranarray(L), np.asfortranarray(B), np.asfortranarray(Xp),
                                1.0 + 0j if cplx else 1.0)
    r = np.abs(L[:, 2]) * delta  # residual column 1 = L[:, 2] * delta
    num = math.sqrt(float(sum(Fraction(float(v)) ** 2 for v in r)))
    den = np.linalg.norm(L) * np.linalg.norm(Xp) + np.linalg.norm(B)
    assert abs(eta - num / den) <= 1e-12 * (num / den)


def test_forward_error_definition():
    Xref = np.array([[3.0, 0.0], [0.0, 4.0]])
    X = Xref + np.array([[0.0, 0.0], [0.0, 0.5]])
    assert oracle.forward_error(X, Xref) == pytest.approx(0.1)


def test_batch_matches_single():
    ms, ns = I.batched_sizes(0, 12)
    As = [I.gen_A(0, int(m), I.C128, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(0, int(m), int(n), I.C128, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    alpha = 1.5 - 0.5j
    Xs = oracle.solve_batch(As, Bs, alpha)
    for A, B, X in zip(As, Bs, Xs):
        assert np.array_equal(X, oracle.solve(A, B, alpha))


def test_cols_match_full():
    A = I.gen_A(0, 200, I.R64)
    B = I.gen_B(0, 200, 31, I.R64)
    X = oracle.solve(A, B, 1.0)
    cols = [0, 5, 30, 17]
    assert np.array_equal(oracle.solve_cols(A, B, 1.0, cols), X[:, cols])


def test_threads_do_not_change_results():
    A = I.gen_A(3, 150, I.C128)
    B = I.gen_B(3, 150, 40, I.C128)
    t0 = oracle.num_threads()
    try:
        oracle.set_num_threads(1)
        X1 = oracle.solve(A, B, 2 - 1j)
        oracle.set_num_threads(max(2, t0))
        X2 = oracle.solve(A, B, 2 - 1j)
    finally:
        oracle.set_num_threads(t0)
    assert np.array_equal(X1, X2)


def test_argument_errors():
    A = np.asfortranarray(np.eye(4))
    with pytest.raises(ValueError):
        oracle.solve(A, np.asfortranarray(np.zeros((3, 2))), 1.0)  # ldb < m
    X = oracle.solve(A, np.asfortranarray(np.zeros((4, 0))), 1.0)  # n = 0 quick return
    assert X.shape == (4, 0)
