"""The fused varlen LU-factor solve (hsma_getrs_vbatched): X = U^{-1} L^{-1} P^T (alpha B)
per instance in one launch, against the oracle's getrs on the same factors; without
pivots it equals the two-launch path (unit lower, then upper) bit for bit.

Factors: scipy's getrf of A = Q (G / sqrt(m) + 2 I) with Q a random row permutation, so the
factorisation interchanges rows and L, U stay well conditioned (forward error of the two
triangular solves ~ m u cond: tolerance 1e-12 for FP64, 2e-5 for FP32 as for the solve)."""
import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu
la = pytest.importorskip("scipy.linalg")


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _instances(seed, batch, cx, lo=1, hi=64):
    ms, ns = I.batched_sizes(seed, batch, lo=lo, hi=hi)
    rng = np.random.default_rng(seed)
    LUs, pivs, Bs = [], [], []
    for m, n in zip(ms, ns):
        m, n = int(m), int(n)
        G = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cx else 0.0)
        A = (G / np.sqrt(m) + 2.0 * np.eye(m))[rng.permutation(m)]
        lu, piv = la.lu_factor(A)
        LUs.append(np.asfortranarray(lu))
        pivs.append((piv + 1).astype(np.int32))
        Bs.append(np.asfortranarray(rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cx else 0.0)))
    return LUs, pivs, Bs


def _run(H, code, LUs, pivs, Bs, alpha, null_every=0):
    """One hsma_getrs_vbatched call; pivs None = no interchanges; null_every k > 0 gives every
    k-th instance a NULL pivot pointer."""
    import torch
    bt = U.Batch(LUs, Bs)
    d_ipiv = 0
    if pivs is not None:
        flat = np.concatenate(pivs).astype(np.int32)
        off = np.concatenate([[0], np.cumsum([len(p) for p in pivs])[:-1]]).astype(np.int64)
        dpiv = torch.from_numpy(flat).cuda()
        ptrs = dpiv.data_ptr() + 4 * off
        if null_every:
            ptrs[::null_every] = 0
        dptr = torch.from_numpy(ptrs.astype(np.int64)).cuda()
        d_ipiv = dptr.data_ptr()
        bt._keep = (dpiv, dptr)
    a = bt.args()
    H.hsma_getrs_vbatched(code, bt.batch, a[0], a[1], alpha, a[2], a[3], d_ipiv, a[4], a[5], max_m=64,
                          d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    return bt


@pytest.mark.parametrize("cx", [False, True])
def test_getrs_batch_matches_oracle(H, cx):
    code = I.C128 if cx else I.R64
    alpha = 1.5 - 0.5j if cx else 0.75
    LUs, pivs, Bs = _instances(31, 700, cx)
    bt = _run(H, code, LUs, pivs, Bs, alpha)
    assert bt.status() == 0
    out = bt.results()
    for b in range(len(LUs)):
        ref = oracle.getrs(LUs[b], pivs[b], Bs[b], alpha)
        assert oracle.forward_error(out[b], ref) <= 1e-12, b


def test_getrs_without_pivots_equals_two_launches(H):
    import torch
    LUs, _, Bs = _instances(32, 500, True, lo=8)
    alpha = 0.5 + 2.0j
    fused = _run(H, I.C128, LUs, None, Bs, alpha).results()
    bt = U.Batch(LUs, Bs)
    a = bt.args()
    H.hsma_trsm_vbatched(I.C128, H.LEFT, H.LOWER, H.NO_TRANS, H.UNIT, bt.batch, a[0], a[1], alpha, a[2], a[3], a[4],
                         a[5], 64, 64, 0, H.stream_ptr())
    H.hsma_trsm_vbatched(I.C128, H.LEFT, H.UPPER, H.NO_TRANS, H.NON_UNIT, bt.batch, a[0], a[1], 1.0, a[2], a[3],
                         a[4], a[5], 64, 64, 0, H.stream_ptr())
    torch.cuda.synchronize()
    two = bt.results()
    for b in range(len(LUs)):
        assert np.array_equal(fused[b], two[b]), b
        assert oracle.forward_error(fused[b], oracle.getrs(LUs[b], None, Bs[b], alpha)) <= 1e-12, b


@pytest.mark.parametrize("cx", [False, True])
def test_getrs_null_pivot_entries_and_alone(H, cx):
    """NULL pivot pointers mean no interchanges for that instance; an instance alone equals it
    in the mix, bit for bit (complex128: the interchange pass's permutation gather)."""
    code = I.C128 if cx else I.R64
    LUs, pivs, Bs = _instances(33, 300, cx)
    mix = _run(H, code, LUs, pivs, Bs, -1.25, null_every=3).results()
    for b in range(len(LUs)):
        ref = oracle.getrs(LUs[b], None if b % 3 == 0 else pivs[b], Bs[b], -1.25)
        assert oracle.forward_error(mix[b], ref) <= 1e-12, b
    for b in range(1, len(LUs), 41):  # alone = in the mix, bit for bit
        alone = _run(H, code, [LUs[b]], None if b % 3 == 0 else [pivs[b]], [Bs[b]], -1.25).results()[0]
        assert np.array_equal(alone, mix[b]), b


def test_getrs_bad_pivot_flagged_and_untouched(H):
    LUs, pivs, Bs = _instances(34, 40, True, lo=4)
    bad = [5, 17]
    for b in bad:
        pivs[b] = pivs[b].copy()
        pivs[b][1] = 1  # row 2 interchanged with row 1: below k, invalid
    bt = _run(H, I.C128, LUs, pivs, Bs, 1.0)
    assert bt.status() & H.DEVERR_BAD_PIVOT
    out = bt.results()
    for b in range(len(LUs)):
        if b in bad:
            assert np.array_equal(out[b], Bs[b]), b
        else:
            assert oracle.forward_error(out[b], oracle.getrs(LUs[b], pivs[b], Bs[b], 1.0)) <= 1e-12, b


@pytest.mark.parametrize("cx", [False, True])
def test_getrs_fp32_dtypes(H, cx):
    code = 5 if cx else 4
    LUs, pivs, Bs = _instances(35, 300, cx)
    t = np.complex64 if cx else np.float32
    LU32 = [np.asfortranarray(x.astype(t)) for x in LUs]
    B32 = [np.asfortranarray(x.astype(t)) for x in Bs]
    out = _run(H, code, LU32, pivs, B32, 1.5).results()
    wide = np.complex128 if cx else np.float64
    for b in range(len(LUs)):
        ref = oracle.getrs(np.asfortranarray(LU32[b].astype(wide)), pivs[b], np.asfortranarray(B32[b].astype(wide)),
                           1.5)
        assert oracle.forward_error(out[b].astype(wide), ref) <= 2e-5, b


@pytest.mark.parametrize("cx", [False, True])
def test_getrs_alpha_zero_and_empty_instances(H, cx):
    """alpha = 0 gives X = 0 (complex128: the interchange pass, then one packed launch writing
    zeros; the second is skipped); empty instances (m = 0, n = 0) are valid no-ops."""
    LUs, pivs, Bs = _instances(36, 30, cx)
    dt = np.complex128 if cx else np.float64
    LUs[3], pivs[3], Bs[3] = np.zeros((0, 0), dt), np.zeros(0, np.int32), np.zeros((0, 0), dt)
    Bs[4] = np.zeros((LUs[4].shape[0], 0), dt)
    bt = _run(H, I.C128 if cx else I.R64, LUs, pivs, Bs, 0.0)
    assert bt.status() == 0
    out = bt.results()
    for b in range(len(LUs)):
        assert out[b].shape == Bs[b].shape and np.all(out[b] == 0.0), b



def _chol_instances(seed, batch, cx, lo=1):
    ms, ns = I.batched_sizes(seed, batch, lo=lo)
    rng = np.random.default_rng(seed)
    Ls, Bs = [], []
    for m, n in zip(ms, ns):
        m, n = int(m), int(n)
        G = rng.standard_normal((m, m)) + (1j * rng.standard_normal((m, m)) if cx else 0.0)
        Lf = la.cholesky(G @ G.conj().T / m + np.eye(m), lower=True)
        Lf[np.triu_indices(m, 1)] = np.nan  # never read
        Ls.append(np.asfortranarray(Lf))
        Bs.append(np.asfortranarray(rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cx else 0.0)))
    return Ls, Bs


def _run_potrs(H, code, Ls, Bs, alpha):
    import torch
    bt = U.Batch(Ls, Bs)
    a = bt.args()
    H.hsma_potrs_vbatched(code, bt.batch, a[0], a[1], alpha, a[2], a[3], a[4], a[5], max_m=64,
                          d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    return bt


@pytest.mark.parametrize("cx", [False, True])
def test_potrs_batch_matches_oracle_and_two_launches(H, cx):
    import torch
    code = I.C128 if cx else I.R64
    alpha = 0.5 - 1.0j if cx else 2.0
    Ls, Bs = _chol_instances(41, 500, cx)
    bt = _run_potrs(H, code, Ls, Bs, alpha)
    assert bt.status() == 0
    fused = bt.results()
    two = U.Batch(Ls, Bs)
    a = two.args()
    H.hsma_trsm_vbatched(code, H.LEFT, H.LOWER, H.NO_TRANS, H.NON_UNIT, two.batch, a[0], a[1], alpha, a[2], a[3],
                         a[4], a[5], 64, 64, 0, H.stream_ptr())
    H.hsma_trsm_vbatched(code, H.LEFT, H.LOWER, H.CONJ_TRANS if cx else H.TRANS, H.NON_UNIT, two.batch, a[0], a[1],
                         1.0, a[2], a[3], a[4], a[5], 64, 64, 0, H.stream_ptr())
    torch.cuda.synchronize()
    two = two.results()
    for b in range(len(Ls)):
        assert np.array_equal(fused[b], two[b]), b
        ref = oracle.potrs(Ls[b], Bs[b], alpha)
        assert oracle.forward_error(fused[b], ref) <= 1e-12, b


def test_potrs_complex64(H):
    Ls, Bs = _chol_instances(42, 200, True)
    L32 = [np.asfortranarray(x.astype(np.complex64)) for x in Ls]
    B32 = [np.asfortranarray(x.astype(np.complex64)) for x in Bs]
    out = _run_potrs(H, 5, L32, B32, 1.0).results()
    for b in range(len(Ls)):
        ref = oracle.potrs(np.asfortranarray(L32[b].astype(np.complex128)), np.asfortranarray(B32[b].astype(np.complex128)), 1.0)
        assert oracle.forward_error(out[b].astype(np.complex128), ref) <= 2e-5, b
