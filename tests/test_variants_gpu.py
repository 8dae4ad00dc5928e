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


def _batch(H, code, uplo, trans, unit, As, Bs, alpha):
    import torch
    bt = U.Batch(As, Bs)
    H.hsma_trsm_vbatched(code, 0, uplo, trans, int(unit), bt.batch, bt.args()[0], bt.args()[1], alpha,
                         bt.args()[2], bt.args()[3], bt.args()[4], bt.args()[5], max_m=64,
                         d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    assert bt.status() == 0
    return bt.results()


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("uplo,trans,unit", [v[1:] for v in VARIANTS if v[0] == 0])
def test_batched_left_variants(H, code, uplo, trans, unit):
    """The varlen batch reads A and B through an index map: every left-side variant equals the
    oracle's definition per instance, and an instance alone equals it in the mix, bit for bit."""
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    ms, ns = I.batched_sizes(13 + uplo + 2 * trans, 160)
    As, Bs = [], []
    for b, (m, n) in enumerate(zip(ms, ns)):
        L = I.gen_A(13, int(m), code, inst=b)
        As.append(np.asfortranarray(L if uplo == 0 else L.T.copy()))
        Bs.append(I.gen_B(13, int(m), int(n), code, inst=b))
    mix = _batch(H, code, uplo, trans, unit, As, Bs, alpha)
    for b in range(len(As)):
        ref = oracle.solve_general(As[b], Bs[b], alpha, 0, uplo, trans, unit)
        assert oracle.forward_error(mix[b], ref) <= 1e-12, b
    for b in range(0, len(As), 23):
        assert np.array_equal(_batch(H, code, uplo, trans, unit, [As[b]], [Bs[b]], alpha)[0], mix[b])


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_batched_lu_solve(H, code):
    """LU-factor solve (the paper's motivating use): packed factors P = tril(L, -1) + triu(U);
    X = U^{-1} L^{-1} (alpha B) as two batched launches, unit lower then upper."""
    alpha = 2.0 if code == I.R64 else 1.0 + 1.0j
    ms, ns = I.batched_sizes(31, 300)
    Ps, Bs = [], []
    for b, (m, n) in enumerate(zip(ms, ns)):
        Lf = I.gen_A(31, int(m), code, inst=b)
        Uf = I.gen_A(32, int(m), code, inst=b).T
        Ps.append(np.asfortranarray(np.tril(Lf, -1) + np.triu(Uf)))
        Bs.append(I.gen_B(31, int(m), int(n), code, inst=b))
    Y = _batch(H, code, 0, 0, True, Ps, Bs, alpha)
    X = _batch(H, code, 1, 0, False, Ps, [np.asfortranarray(y) for y in Y], 1.0)
    for b in range(len(Ps)):
        ref = oracle.solve_general(Ps[b], oracle.solve_general(Ps[b], Bs[b], alpha, 0, 0, 0, True), 1.0, 0, 1, 0,
                                   False)
        assert oracle.forward_error(X[b], ref) <= 1e-12, b
