"""Pins for the oracle's LU-factor solve (getrs), by means other than the oracle itself:
LAPACK's getrs (scipy.linalg.lu_solve, a black box) on getrf factors; the residual of
P L U X = alpha B with A rebuilt from the factors; L = U = I, where X = P^T (alpha B)
exactly; and the interchanges written out as a permutation matrix."""
import numpy as np
import pytest

import oracle

la = pytest.importorskip("scipy.linalg")


def _factors(seed, m, cx):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cx else 0.0)
    lu, piv = la.lu_factor(A)
    return np.asfortranarray(A), np.asfortranarray(lu), piv + 1  # LAPACK's 1-based pivots


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("m,n", [(1, 3), (7, 5), (33, 17), (64, 64)])
def test_getrs_matches_lapack_and_residual(cx, m, n):
    A, LU, ipiv = _factors(m * 7 + n, m, cx)
    rng = np.random.default_rng(m)
    B = np.asfortranarray(rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cx else 0.0))
    alpha = 0.75 - 1.5j if cx else -1.25
    X = oracle.getrs(LU, ipiv, B, alpha)
    ref = la.lu_solve((LU, ipiv - 1), alpha * B)
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)
    R = A @ X - alpha * B
    assert np.linalg.norm(R) <= 1e-12 * (np.linalg.norm(A) * np.linalg.norm(X) + abs(alpha) * np.linalg.norm(B))


def test_getrs_identity_factors_is_the_permutation():
    m, n = 9, 4
    ipiv = np.array([3, 2, 9, 5, 5, 8, 7, 8, 9])  # 1-based, ipiv[k] >= k + 1
    LU = np.asfortranarray(np.eye(m))
    B = np.asfortranarray(np.arange(m * n, dtype=np.float64).reshape(m, n, order="F"))
    X = oracle.getrs(LU, ipiv, B, 2.0)
    P = np.eye(m)
    for k, p in enumerate(ipiv - 1):  # P^T as the product of the interchanges
        P[[k, p], :] = P[[p, k], :]
    assert np.array_equal(X, P @ (2.0 * B))


def test_getrs_without_pivots_is_two_triangular_solves():
    A, LU, _ = _factors(3, 20, True)
    B = np.asfortranarray(np.ones((20, 3), dtype=np.complex128))
    X = oracle.getrs(LU, None, B, 1.0)
    L = np.tril(LU, -1) + np.eye(20)
    U = np.triu(LU)
    ref = la.solve_triangular(U, la.solve_triangular(L, B, lower=True, unit_diagonal=True), lower=False)
    assert np.linalg.norm(X - ref) <= 1e-13 * np.linalg.norm(ref)


def test_getrs_rejects_pivot_out_of_range():
    with pytest.raises(ValueError):
        oracle.getrs(np.asfortranarray(np.eye(3)), np.array([2, 1, 3]), np.asfortranarray(np.ones((3, 1))), 1.0)


def _chol(seed, m, cx):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cx else 0.0)
    A = G @ G.conj().T / m + np.eye(m)
    return np.asfortranarray(A), np.asfortranarray(la.cholesky(A, lower=True))


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("m,n", [(1, 2), (9, 4), (40, 31), (64, 64)])
def test_potrs_matches_lapack_and_residual(cx, m, n):
    A, Lf = _chol(m + 100 * n, m, cx)
    P = Lf.copy(order="F")
    P[np.triu_indices(m, 1)] = np.nan  # the strict upper triangle is never read
    rng = np.random.default_rng(n)
    B = np.asfortranarray(rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cx else 0.0))
    alpha = 1.25 + 0.5j if cx else 0.5
    X = oracle.potrs(P, B, alpha)
    ref = la.cho_solve((Lf, True), alpha * B)
    assert np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)
    R = A @ X - alpha * B
    assert np.linalg.norm(R) <= 1e-12 * (np.linalg.norm(A) * np.linalg.norm(X) + abs(alpha) * np.linalg.norm(B))


GETRS_MUTANTS = {
    "interchanges applied in reverse order": (
        "for k, p in enumerate(np.asarray(ipiv, dtype=np.int64)):",
        "for k, p in reversed(list(enumerate(np.asarray(ipiv, dtype=np.int64)))):"),
    "unit diagonal of L ignored": ("Y = solve_general(LU, Y, alpha, 0, 0, 0, True, _lib=_lib)",
                                   "Y = solve_general(LU, Y, alpha, 0, 0, 0, False, _lib=_lib)"),
    "upper factor read as lower": ("return solve_general(LU, Y, 1.0, 0, 1, 0, False, _lib=_lib)",
                                   "return solve_general(LU, Y, 1.0, 0, 0, 0, False, _lib=_lib)"),
}
POTRS_MUTANTS = {
    "second solve not transposed": ("return solve_general(Lf, Y, 1.0, 0, 0, 2 if np.iscomplexobj(Lf) else 1, False,",
                                    "return solve_general(Lf, Y, 1.0, 0, 0, 0, False,"),
    "transposed without conjugation": ("0, 0, 2 if np.iscomplexobj(Lf) else 1, False,", "0, 0, 1, False,"),
}


def _mutant(fn, old, new):
    import inspect
    src = inspect.getsource(fn)
    assert src.count(old) == 1, f"mutation site not found: {old}"
    ns = dict(vars(oracle))
    exec(src.replace(old, new, 1), ns)
    return ns[fn.__name__]


@pytest.mark.parametrize("name", list(GETRS_MUTANTS))
def test_getrs_pins_catch_mutant(name):
    bad = _mutant(oracle.getrs, *GETRS_MUTANTS[name])
    caught = False
    for cx in (False, True):
        A, LU, ipiv = _factors(17, 33, cx)
        B = np.asfortranarray(np.arange(33 * 4, dtype=np.float64).reshape(33, 4) - 50.0)
        if cx:
            B = np.asfortranarray(B + 0.5j * B[::-1])
        X = bad(LU, ipiv, B, 1.0)
        ref = la.lu_solve((LU, ipiv - 1), B)
        caught |= not np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref)
    assert caught, name


@pytest.mark.parametrize("name", list(POTRS_MUTANTS))
def test_potrs_pins_catch_mutant(name):
    bad = _mutant(oracle.potrs, *POTRS_MUTANTS[name])
    A, Lf = _chol(5, 20, True)
    B = np.asfortranarray(np.arange(60, dtype=np.float64).reshape(20, 3) * (1 - 0.5j))
    X = bad(Lf, B, 1.0)
    ref = la.cho_solve((Lf, True), B)
    assert not np.linalg.norm(X - ref) <= 1e-12 * np.linalg.norm(ref), name
