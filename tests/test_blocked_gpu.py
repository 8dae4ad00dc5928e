"""Blocked large-case path (Section 4.3) against the oracle, through the C ABI."""
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


def _dt(code):
    return np.float64 if code == I.R64 else np.complex128


def _run(H, code, A, B, alpha, nb, unit=False, **cfg):
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    opts = H.Opts()
    opts.path = H.PATH_BLOCKED
    opts.nb = nb
    for k, v in cfg.items():
        setattr(opts, k, v)
    info = H.Info()
    H.hsma_trsm_llnn_ex(code, int(unit), A.shape[1], B.shape[1], alpha, dA.data_ptr(), A.shape[0], dB.data_ptr(),
                        B.shape[0], H.stream_ptr(), opts=opts, info=info)
    torch.cuda.synchronize()
    assert info.plan.path == H.PATH_BLOCKED and info.plan.nb == nb
    return H.from_device(dB)


CASES = [(65, 7, 32), (127, 64, 64), (128, 1, 64), (129, 33, 128), (300, 200, 128), (1000, 100, 256),
         (700, 50, 512), (2048, 300, 256), (96, 97, 32), (513, 5, 512)]


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("pad", [0, 3])
@pytest.mark.parametrize("m,n,nb", CASES)
def test_blocked_parity(H, code, m, n, nb, pad):
    """Ragged sizes, every N_B, leading dimensions with (pad 0, even m) and without TMA (odd fp64 ld)."""
    alpha = 1.0 if code == I.R64 else 1.5 - 0.5j
    seed = m * 7 + n
    A0, B0 = I.gen_A(seed, m, code), I.gen_B(seed, m, n, code)
    A = I.embed(A0, m + pad, fill=np.nan)
    A[:m][np.triu_indices(m, 1)] = np.nan  # the strict upper triangle is never read
    B = I.embed(B0, m + pad, fill=np.nan)
    X = _run(H, code, A, B, alpha, nb)
    assert np.all(np.isnan(X[m:])), "padding rows written"
    ref = oracle.solve(A0, B0, alpha)
    err = oracle.forward_error(X[:m], ref)
    assert err <= TOL, err
    assert H.hsma_device_status() == 0


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_blocked_unit_diagonal_and_alpha(H, code):
    m, n, nb = 333, 41, 128
    A0, B0 = I.gen_A(2, m, code), I.gen_B(2, m, n, code)
    A = np.array(A0, order="F")
    np.fill_diagonal(A, np.nan)
    alpha = -0.75 if code == I.R64 else 0.25 + 1j
    X = _run(H, code, A, B0, alpha, nb, unit=True)
    A1 = np.array(A0, order="F")
    np.fill_diagonal(A1, 1.0)
    assert oracle.forward_error(X, oracle.solve(A1, B0, alpha)) <= TOL
    # alpha = 0 on the blocked path: B := 0, A not read
    Anan = np.full((m, m), np.nan, dtype=_dt(code), order="F")
    X0 = _run(H, code, Anan, B0, 0.0, nb)
    assert np.all(X0 == 0)


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_planner_default_matches_oracle(H, code):
    """hsma_trsm_llnn with the planner's own N_B (the table lookup of Section 4.3.2)."""
    import torch
    m, n = 777, 129
    A, B = I.gen_A(4, m, code), I.gen_B(4, m, n, code)
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    dA, dB = H.to_device(A), H.to_device(B)
    H.hsma_trsm_llnn(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
    torch.cuda.synchronize()
    X = H.from_device(dB)
    assert oracle.forward_error(X, oracle.solve(A, B, alpha)) <= TOL
    assert oracle.backward_error(A, B, X, alpha) <= 1e-14


CFG_CASES = [(65, 7, 32), (300, 200, 128), (700, 50, 512), (1000, 9, 64), (513, 130, 256)]


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("looking", [1, 2], ids=["right", "left"])
@pytest.mark.parametrize("tile", [1, 2, 3], ids=["64x64", "128x16", "128x8"])
@pytest.mark.parametrize("split_k", [1, 2], ids=["split", "nosplit"])
@pytest.mark.parametrize("m,n,nb", CFG_CASES)
def test_blocked_configurations_parity(H, code, looking, tile, split_k, m, n, nb):
    """Every configuration the autotuner may choose (update direction, product tile, split
    K) at ragged sizes, with NaN in the never-read upper triangle and padding rows."""
    import torch
    alpha = 1.25 if code == I.R64 else 0.5 - 1.5j
    seed = m + 3 * n + nb
    A0, B0 = I.gen_A(seed, m, code), I.gen_B(seed, m, n, code)
    A = I.embed(A0, m + 2, fill=np.nan)
    A[:m][np.triu_indices(m, 1)] = np.nan
    B = I.embed(B0, m + 2, fill=np.nan)
    X = _run(H, code, A, B, alpha, nb, looking=looking, tile=tile, split_k=split_k)
    assert np.all(np.isnan(X[m:]))
    assert oracle.forward_error(X[:m], oracle.solve(A0, B0, alpha)) <= TOL
    assert H.hsma_device_status() == 0


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_left_looking_unit_diagonal(H, code):
    m, n, nb = 450, 33, 64
    A0, B0 = I.gen_A(6, m, code), I.gen_B(6, m, n, code)
    A = np.array(A0, order="F")
    np.fill_diagonal(A, np.nan)
    X = _run(H, code, A, B0, -2.0, nb, unit=True, looking=2)
    A1 = np.array(A0, order="F")
    np.fill_diagonal(A1, 1.0)
    assert oracle.forward_error(X, oracle.solve(A1, B0, -2.0)) <= TOL
