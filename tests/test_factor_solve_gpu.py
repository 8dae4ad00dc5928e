"""One solve with LU or Cholesky factors at any m (hsma_getrs, hsma_potrs): the
interchanges, then the two triangular solves through the small kernel (m <= 64) or
the blocked path, against the oracle's getrs / potrs.  Factors from scipy's getrf /
potrf of well-conditioned matrices (rows permuted, so getrf interchanges rows)."""
import numpy as np
import pytest

import oracle
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
la = pytest.importorskip("scipy.linalg")


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _mat(rng, m, n, cx):
    return rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cx else 0.0)


def _lu(seed, m, n, cx):
    rng = np.random.default_rng(seed)
    A = (_mat(rng, m, m, cx) / np.sqrt(m) + 2.0 * np.eye(m))[rng.permutation(m)]
    lu, piv = la.lu_factor(A)
    return np.asfortranarray(lu), (piv + 1).astype(np.int32), np.asfortranarray(_mat(rng, m, n, cx))


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("m,n,emulated", [(37, 20, 0), (64, 64, 0), (300, 50, 0), (1000, 33, 0), (700, 40, 1)])
def test_getrs_single(H, cx, m, n, emulated):
    import torch
    code = 1 if cx else 0
    alpha = 1.5 - 0.5j if cx else -0.75
    LU, ipiv, B = _lu(m * 3 + n, m, n, cx)
    dLU, dB = H.to_device(LU), H.to_device(B)
    dpiv = torch.from_numpy(ipiv).cuda()
    opts = H.Opts()
    opts.fp64_products = emulated
    H.hsma_getrs(code, m, n, alpha, dLU.data_ptr(), m, dpiv.data_ptr(), dB.data_ptr(), m, H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    X = H.from_device(dB)
    assert oracle.forward_error(X, oracle.getrs(LU, ipiv, B, alpha)) <= 1e-12


def test_getrs_single_bad_pivot_flagged(H):
    import torch
    LU, ipiv, B = _lu(5, 40, 3, False)
    ipiv[7] = 2  # row 8 interchanged with row 2: below k
    dLU, dB = H.to_device(LU), H.to_device(B)
    dpiv = torch.from_numpy(ipiv).cuda()
    H.hsma_getrs(0, 40, 3, 1.0, dLU.data_ptr(), 40, dpiv.data_ptr(), dB.data_ptr(), 40, H.stream_ptr())
    torch.cuda.synchronize()
    assert H.hsma_device_status() & H.DEVERR_BAD_PIVOT
    # the interchanges were skipped: the result is the unpermuted solve
    assert oracle.forward_error(H.from_device(dB), oracle.getrs(LU, None, B, 1.0)) <= 1e-12


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("m,n", [(50, 7), (257, 64), (900, 20)])
def test_potrs_single(H, cx, m, n):
    import torch
    rng = np.random.default_rng(m + n)
    G = _mat(rng, m, m, cx)
    Lf = la.cholesky(G @ G.conj().T / m + np.eye(m), lower=True)
    Lf[np.triu_indices(m, 1)] = np.nan  # not read
    Lf = np.asfortranarray(Lf)
    B = np.asfortranarray(_mat(rng, m, n, cx))
    alpha = 0.25 + 2.0j if cx else 3.0
    dL, dB = H.to_device(Lf), H.to_device(B)
    H.hsma_potrs(1 if cx else 0, m, n, alpha, dL.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    assert oracle.forward_error(H.from_device(dB), oracle.potrs(Lf, B, alpha)) <= 1e-12


@pytest.mark.parametrize("code,m,n", [(0, 64, 1), (1, 200, 3), (3, 300, 20)])
def test_getrs_single_without_pivots(H, code, m, n):
    """ipiv = NULL: no interchanges; dtype 3 runs each triangular solve in the FP64-result
    refinement mode."""
    import torch
    cx = code == 1
    LU, _, B = _lu(m + 7 * n, m, n, cx)
    dLU, dB = H.to_device(LU), H.to_device(B)
    H.hsma_getrs(code, m, n, 1.25, dLU.data_ptr(), m, 0, dB.data_ptr(), m, H.stream_ptr())
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    assert oracle.forward_error(H.from_device(dB), oracle.getrs(LU, None, B, 1.25)) <= 1e-12


def test_potrs_single_emulated_products(H):
    import torch
    m, n = 700, 30
    rng = np.random.default_rng(7)
    G = _mat(rng, m, m, False)
    Lf = np.asfortranarray(la.cholesky(G @ G.T / m + np.eye(m), lower=True))
    B = np.asfortranarray(_mat(rng, m, n, False))
    dL, dB = H.to_device(Lf), H.to_device(B)
    opts = H.Opts()
    opts.fp64_products = 1
    H.hsma_potrs(0, m, n, 1.0, dL.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    assert oracle.forward_error(H.from_device(dB), oracle.potrs(Lf, B, 1.0)) <= 1e-12
