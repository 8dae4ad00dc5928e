"""Native FP32 and complex64 dtypes (HSMA_R32, HSMA_C64): the small direct solve
and the varlen batch compute in FP32; larger m runs the FP32-result blocked
solve (R32) or a complex128 emulated-FP64 solve rounded back (C64).

Reference: the FP64 oracle applied to the same FP32 inputs (widened exactly).
Tolerance 2e-5 relative Frobenius forward error: FP32 substitution errs by at
most about m u_32 cond(L) (m <= 64, u_32 = 6e-8, cond <= 2 for these
generators: < 8e-6), and the blocked FP32-result path is held to the same
bound as HSMA_R32_BF16."""
import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _f32(code64, X):
    return np.asfortranarray(X.astype(np.float32 if code64 == I.R64 else np.complex64))


def _solve(H, code, A, B, alpha, unit=False, opts=None):
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    m, n = B.shape
    H.hsma_trsm_llnn_ex(code, int(unit), A.shape[1], n, alpha, dA.data_ptr(), A.shape[0], dB.data_ptr(), m,
                        H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    return H.from_device(dB)


def _ref(A32, B32, alpha, unit=False):
    wide = np.complex128 if np.iscomplexobj(A32) else np.float64
    return oracle.solve(np.asfortranarray(A32.astype(wide)), np.asfortranarray(B32.astype(wide)), alpha, unit=unit)


@pytest.mark.parametrize("code64,code", [(I.R64, 4), (I.C128, 5)])
@pytest.mark.parametrize("n", [1, 5, 33, 64])
def test_small_fp32_every_m(H, code64, code, n):
    alpha = 1.5 if code64 == I.R64 else 1.5 - 0.5j
    for m in list(range(1, 65, 3)) + [64]:
        A32, B32 = _f32(code64, I.gen_A(m, m, code64)), _f32(code64, I.gen_B(m, m, n, code64))
        X = _solve(H, code, A32, B32, alpha)
        assert X.dtype == A32.dtype
        err = oracle.forward_error(X.astype(np.complex128 if code == 5 else np.float64), _ref(A32, B32, alpha))
        assert err <= TOL32, (m, err)


@pytest.mark.parametrize("code64,code", [(I.R64, 4), (I.C128, 5)])
def test_small_fp32_unit_diagonal_not_read(H, code64, code):
    m, n = 40, 17
    A32, B32 = _f32(code64, I.gen_A(3, m, code64)), _f32(code64, I.gen_B(3, m, n, code64))
    A = A32.copy(order="F")
    A[np.diag_indices(m)] = np.nan
    X = _solve(H, code, A, B32, 1.0, unit=True)
    assert np.all(np.isfinite(X))
    assert oracle.forward_error(X.astype(np.complex128 if code == 5 else np.float64),
                                _ref(A32, B32, 1.0, unit=True)) <= TOL32


@pytest.mark.parametrize("code64,code", [(I.R64, 4), (I.C128, 5)])
def test_batched_fp32_parity_and_alone(H, code64, code):
    import torch
    alpha = 1.5 if code64 == I.R64 else 1.5 - 0.5j
    ms, ns = I.batched_sizes(21, 600)
    As = [_f32(code64, I.gen_A(21, int(m), code64, inst=b)) for b, m in enumerate(ms)]
    Bs = [_f32(code64, I.gen_B(21, int(m), int(n), code64, inst=b)) for b, (m, n) in enumerate(zip(ms, ns))]

    def run(As_, Bs_):
        bt = U.Batch(As_, Bs_)
        H.hsma_trsm_llnn_vbatched(code, 0, bt.batch, bt.args()[0], bt.args()[1], alpha, bt.args()[2],
                                  bt.args()[3], bt.args()[4], bt.args()[5], max_m=64, max_n=0,
                                  d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
        torch.cuda.synchronize()
        assert bt.status() == 0
        return bt.results()
    mix = run(As, Bs)
    wide = np.complex128 if code == 5 else np.float64
    for b in range(len(As)):
        assert oracle.forward_error(mix[b].astype(wide), _ref(As[b], Bs[b], alpha)) <= TOL32, b
    for b in range(0, len(As), 37):
        assert np.array_equal(run([As[b]], [Bs[b]])[0], mix[b]), b


@pytest.mark.parametrize("code64,code", [(I.R64, 4), (I.C128, 5)])
@pytest.mark.parametrize("m,n", [(65, 7), (300, 100), (1000, 64)])
def test_blocked_fp32_dtypes(H, code64, code, m, n):
    alpha = 1.0 if code64 == I.R64 else 1.5 - 0.5j
    A32, B32 = _f32(code64, I.gen_A(m + 1, m, code64)), _f32(code64, I.gen_B(m + 1, m, n, code64))
    A = A32.copy(order="F")
    A[np.triu_indices(m, 1)] = np.nan  # only the lower triangle is read
    X = _solve(H, code, A, B32, alpha)
    wide = np.complex128 if code == 5 else np.float64
    assert oracle.forward_error(X.astype(wide), _ref(A32, B32, alpha)) <= TOL32


def test_host_batch_complex64_equals_device_batch(H):
    import torch
    alpha = 0.5 + 2.0j
    ms, ns = I.batched_sizes(4, 300)
    As = [_f32(I.C128, I.gen_A(4, int(m), I.C128, inst=b)) for b, m in enumerate(ms)]
    Bs = [_f32(I.C128, I.gen_B(4, int(m), int(n), I.C128, inst=b)) for b, (m, n) in enumerate(zip(ms, ns))]
    bt = U.Batch(As, Bs)
    H.hsma_trsm_llnn_vbatched(5, 0, bt.batch, bt.args()[0], bt.args()[1], alpha, bt.args()[2], bt.args()[3],
                              bt.args()[4], bt.args()[5], max_m=64, stream=H.stream_ptr())
    torch.cuda.synchronize()
    dev = bt.results()
    m32, n32 = ms.astype(np.int32), ns.astype(np.int32)
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)[:-1]]).astype(np.int64)
    offB = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]]).astype(np.int64)
    hA = np.concatenate([a.ravel(order="F") for a in As])
    hB = np.concatenate([b.ravel(order="F") for b in Bs])
    hX = np.empty_like(hB)
    H.hsma_trsm_llnn_vbatched_host(5, 0, len(As), m32, n32, alpha, hA.ctypes.data, offA, hB.ctypes.data, offB,
                                   hX.ctypes.data, stream=H.stream_ptr())
    torch.cuda.synchronize()
    for b in range(len(As)):
        got = hX[offB[b]:offB[b] + ms[b] * ns[b]].reshape((ms[b], ns[b]), order="F")
        assert np.array_equal(got, dev[b]), b
