"""BLAS triangular-solve variants (side, uplo, trans, diag) through hsma_trsm on the
GPU against the oracle's definition of each variant, small and blocked sizes, every
dtype; the unreferenced triangle is poisoned with NaN."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

VARIANTS = list(itertools.product((0, 1), (0, 1), (0, 1, 2), (False, True)))


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _problem(seed, side, uplo, code, m, n):
    na = m if side == 0 else n
    L = I.gen_A(seed, na, code)
    A = np.asfortranarray(L if uplo == 0 else L.T.copy())
    B = I.gen_B(seed + 1, m, n, code)
    return A, B


def _run(H, code, side, uplo, trans, unit, A, B, alpha, opts=None):
    import torch
    P = A.copy(order="F")
    na = P.shape[0]
    P[np.tril_indices(na, -1) if uplo == 1 else np.triu_indices(na, 1)] = np.nan
    if unit:
        P[np.diag_indices(na)] = np.nan
    dA, dB = H.to_device(P), H.to_device(B)
    m, n = B.shape
    H.hsma_trsm(code, side, uplo, trans, int(unit), m, n, alpha, dA.data_ptr(), na, dB.data_ptr(), m,
                H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    return H.from_device(dB)


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("m,n", [(37, 23), (200, 150)])
@pytest.mark.parametrize("side,uplo,trans,unit", VARIANTS)
def test_variant_parity(H, code, m, n, side, uplo, trans, unit):
    alpha = 1.5 if code == I.R64 else 0.5 - 1.25j
    A, B = _problem(m + 7 * side + 3 * uplo + trans, side, uplo, code, m, n)
    X = _run(H, code, side, uplo, trans, unit, A, B, alpha)
    ref = oracle.solve_general(A, B, alpha, side, uplo, trans, unit)
    assert oracle.forward_error(X, ref) <= 1e-12


@pytest.mark.parametrize("code,code32", [(I.R64, 4), (I.C128, 5)])
@pytest.mark.parametrize("side,uplo,trans", [(1, 0, 0), (0, 1, 1), (1, 1, 2), (0, 0, 2)])
def test_variant_fp32_dtypes(H, code, code32, side, uplo, trans):
    m, n = 60, 90
    A, B = _problem(4, side, uplo, code, m, n)
    f32 = np.float32 if code == I.R64 else np.complex64
    A32, B32 = np.asfortranarray(A.astype(f32)), np.asfortranarray(B.astype(f32))
    X = _run(H, code32, side, uplo, trans, False, A32, B32, 1.0)
    ref = oracle.solve_general(np.asfortranarray(A32.astype(A.dtype)), np.asfortranarray(B32.astype(B.dtype)), 1.0,
                               side, uplo, trans, False)
    assert oracle.forward_error(X.astype(ref.dtype), ref) <= 2e-5


@pytest.mark.parametrize("side,uplo,trans", [(1, 1, 0), (0, 1, 2)])
def test_variant_with_emulated_products(H, side, uplo, trans):
    m, n = 700, 300
    A, B = _problem(9, side, uplo, I.C128, m, n)
    opts = H.Opts()
    opts.fp64_products = 1
    X = _run(H, I.C128, side, uplo, trans, False, A, B, 2.0, opts=opts)
    assert oracle.forward_error(X, oracle.solve_general(A, B, 2.0, side, uplo, trans, False)) <= 1e-12
