"""FP64 products emulated on the BF16 tensor cores: the standalone product
(C -= A X) and the blocked solve with emulated solve and update products
(fp64_products = 1), against exact integer results and the oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _gemm(H, A, X, C):
    import torch
    dA, dX, dC = H.to_device(A), H.to_device(X), H.to_device(C)
    M, K = A.shape
    N = X.shape[1]
    H.hsma_gemm_f64_emulated(M, N, K, dA.data_ptr(), A.shape[0], dX.data_ptr(), X.shape[0], dC.data_ptr(),
                             C.shape[0], H.stream_ptr())
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    return H.from_device(dC)


@pytest.mark.parametrize("M,N,K", [(300, 200, 77), (129, 1, 64), (1000, 513, 1000), (64, 300, 1024)])
def test_emulated_gemm_exact_on_integers(H, M, N, K):
    """Small integers: every product, sum and FP64 update is exact, so the result is bitwise the exact one."""
    rng = np.random.default_rng(M * N + K)
    A = np.asfortranarray(rng.integers(-1024, 1025, (M, K)).astype(np.float64))
    X = np.asfortranarray(rng.integers(-1024, 1025, (K, N)).astype(np.float64))
    C0 = np.asfortranarray(rng.integers(-2 ** 20, 2 ** 20, (M, N)).astype(np.float64))
    got = _gemm(H, A, X, C0)
    exact = C0 - (A.astype(np.int64) @ X.astype(np.int64)).astype(np.float64)
    assert np.array_equal(got, exact)


def _two_prod(a, b):
    """a*b = p + e exactly (Dekker's product with Veltkamp's splitting; |a|, |b| << 2^996)."""
    p = a * b
    f = 134217729.0  # 2^27 + 1

    def split(x):
        c = f * x
        hi = c - (c - x)
        return hi, x - hi
    ah, al = split(a)
    bh, bl = split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


@pytest.mark.parametrize("M,N,K", [(300, 200, 77), (513, 260, 1600), (200, 150, 8192), (130, 257, 16384)])
def test_emulated_gemm_fp64_accuracy(H, M, N, K):
    """Random FP64 data with rows and columns of X scaled over 2^-30..2^30, up to the exactness
    bound K = 2^14.  Sampled entries against the correctly rounded C0 - A X (exact products,
    math.fsum): error within 2^-50 (|C0| + |A||X|), far below one dropped slice pair (~2^-30)."""
    import math
    rng = np.random.default_rng(K)
    A = np.asfortranarray(rng.uniform(-1, 1, (M, K)) * np.exp2(rng.integers(-30, 30, (M, 1))))
    X = np.asfortranarray(rng.uniform(-1, 1, (K, N)) * np.exp2(rng.integers(-30, 30, (1, N))))
    C0 = np.asfortranarray(rng.uniform(-1, 1, (M, N)))
    got = _gemm(H, A, X, C0)
    pick = np.random.default_rng(1)
    rows = np.concatenate([[0, M - 1], pick.integers(0, M, 126)])
    cols = np.concatenate([[N - 1, 0], pick.integers(0, N, 126)])
    for i, j in zip(rows, cols):
        p, e = _two_prod(A[i, :], X[:, j])
        exact = math.fsum(np.concatenate([[C0[i, j]], -p, -e]))
        scale = abs(C0[i, j]) + np.abs(A[i, :]) @ np.abs(X[:, j])
        assert abs(got[i, j] - exact) <= 2.0 ** -50 * scale, (i, j, abs(got[i, j] - exact) / scale)


def test_emulated_gemm_rejects_bad_arguments(H):
    assert H.hsma_gemm_f64_emulated(4, 4, 16385, 1, 4, 1, 16385, 1, 4, 0, check=False) == H.ERR_UNSUPPORTED
    assert H.hsma_gemm_f64_emulated(4, 4, 4, 1, 3, 1, 4, 1, 4, 0, check=False) == H.ERR_INVALID_ARG
    assert H.hsma_gemm_f64_emulated(4, 4, 4, 0, 4, 1, 4, 1, 4, 0, check=False) == H.ERR_INVALID_ARG
    assert H.hsma_gemm_f64_emulated(0, 4, 4, 0, 1, 0, 4, 0, 1, 0, check=False) == H.OK


def _run(H, code, A, B, alpha, nb, unit=False):
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    opts = H.Opts()
    opts.path = H.PATH_BLOCKED
    opts.nb = nb
    opts.fp64_products = 1
    info = H.Info()
    H.hsma_trsm_llnn_ex(code, int(unit), A.shape[1], B.shape[1], alpha, dA.data_ptr(), A.shape[0], dB.data_ptr(),
                        B.shape[0], H.stream_ptr(), opts=opts, info=info)
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    assert info.plan.nb == nb
    return H.from_device(dB)


CASES = [(65, 7, 32), (129, 33, 128), (300, 200, 128), (1000, 100, 256), (700, 50, 512), (2048, 300, 256),
         (96, 97, 64), (513, 1, 512)]


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("pad", [0, 3])
@pytest.mark.parametrize("m,n,nb", CASES)
def test_emulated_blocked_parity(H, code, m, n, nb, pad):
    """Ragged sizes and every N_B; NaN in the upper triangle and in B's padding rows is never read."""
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    seed = m * 11 + n
    A0, B0 = I.gen_A(seed, m, code), I.gen_B(seed, m, n, code)
    A = I.embed(A0, m + pad, fill=np.nan)
    A[:m][np.triu_indices(m, 1)] = np.nan
    B = I.embed(B0, m + pad, fill=np.nan)
    X = _run(H, code, A, B, alpha, nb)
    assert np.all(np.isnan(X[m:])), "padding rows written"
    ref = oracle.solve(A0, B0, alpha)
    err = oracle.forward_error(X[:m], ref)
    assert err <= TOL, err


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_emulated_blocked_unit_diagonal(H, code):
    m, n = 700, 64
    A0, B0 = I.gen_A(5, m, code), I.gen_B(5, m, n, code)
    A = A0.copy(order="F")
    A[np.diag_indices(m)] = np.nan  # not read under UNIT
    X = _run(H, code, A, B0, 1.0, 128, unit=True)
    ref = oracle.solve(A0, B0, 1.0, unit=True)
    assert oracle.forward_error(X, ref) <= TOL


def test_emulated_blocked_badly_scaled_rows(H):
    """Rows of A and B scaled by powers of two from 2^-300 to 2^300: the solution is unchanged
    and the per-row scales of the slices keep it at full accuracy (exponent rebasing falls back
    to ldexp outside the normal range)."""
    m, n = 900, 40
    rng = np.random.default_rng(9)
    A0, B0 = I.gen_A(9, m, I.R64), I.gen_B(9, m, n, I.R64)
    d = np.exp2(rng.integers(-300, 301, m).astype(np.float64))
    A = np.asfortranarray(A0 * d[:, None])
    B = np.asfortranarray(B0 * d[:, None])
    X = _run(H, I.R64, A, B, 1.0, 128)
    ref = oracle.solve(A0, B0, 1.0)
    assert oracle.forward_error(X, ref) <= TOL


@pytest.mark.parametrize("code,m", [(I.R64, 8192), (I.C128, 4096)])
def test_emulated_blocked_large_sampled_columns(H, code, m):
    """Device-generated inputs at a size that spans many block steps; seeded sampled columns
    checked against the oracle's solve of those columns."""
    import torch
    n = 2048
    seed = 3
    dt = torch.float64 if code == I.R64 else torch.complex128
    dA = torch.empty((m, m), dtype=dt, device="cuda")
    dB = torch.empty((n, m), dtype=dt, device="cuda")
    st = H.stream_ptr()
    H.hsma_gen_matrix(code, 0, seed, -1, m, m, dA.data_ptr(), m, st)
    H.hsma_gen_matrix(code, 1, seed, -1, m, n, dB.data_ptr(), m, st)
    opts = H.Opts()
    opts.fp64_products = 1
    H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, st, opts=opts)
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    rng = np.random.default_rng(77)
    cols = np.sort(rng.choice(n, size=32, replace=False))
    cols[0], cols[-1] = 0, n - 1
    got = dB[torch.from_numpy(cols).cuda()].cpu().numpy().T
    A = I.gen_A(seed, m, code)
    ref = oracle.solve(A, I.gen_B_cols(seed, m, cols, code), 1.0)
    errs = [oracle.forward_error(got[:, k], ref[:, k]) for k in range(len(cols))]
    assert max(errs) <= TOL, max(errs)
