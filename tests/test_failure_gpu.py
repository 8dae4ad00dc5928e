"""Failure detection without a GPU fault.

(a) A bounded device wait that runs out: the self-check kernel waits on an
mbarrier nothing arrives on; the wait gives up after its limit, the timeout bit
reaches the host through hsma_device_status, and the context keeps working.
(b) Host-side fault injection: HSMA_FAULT_ALLOC_AFTER=0 makes every workspace
allocation fail; each entry point that allocates returns HSMA_ERR_NO_MEMORY
before it launches anything (B is left as it was), and the same call succeeds
once the injection is off."""
import time

import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _small_solve_ok(H):
    import torch
    A, B = I.gen_A(2, 48, I.R64), I.gen_B(2, 48, 9, I.R64)
    dA, dB = H.to_device(A), H.to_device(B)
    H.hsma_trsm_llnn(I.R64, 0, 48, 9, 1.0, dA.data_ptr(), 48, dB.data_ptr(), 48, H.stream_ptr())
    torch.cuda.synchronize()
    return oracle.forward_error(H.from_device(dB), oracle.solve(A, B, 1.0)) <= 1e-13


@pytest.mark.parametrize("limit_ms", [5, 200])
def test_bounded_wait_runs_out_and_context_survives(H, limit_ms):
    import torch
    assert H.hsma_device_status() == 0
    ret = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    H.hsma_check_wait_timeout(limit_ms * 1_000_000, ret.data_ptr(), H.stream_ptr())
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    assert int(ret.item()) == 2, "the wait did not give up"
    assert wall >= 0.9 * limit_ms / 1e3, wall
    assert H.hsma_device_status() & H.DEVERR_TIMEOUT
    assert H.hsma_device_status() == 0, "error word not cleared by the read"
    assert _small_solve_ok(H), "context unusable after the timeout"
    assert H.hsma_device_status() == 0


def test_wait_check_rejects_bad_arguments(H):
    assert H.hsma_check_wait_timeout(10_000_000, 0, check=False) == H.ERR_INVALID_ARG


def _blocked(H, code, m, n, fp64_products=0):
    def call(dA, dB, check):
        opts = H.Opts()
        opts.path = H.PATH_BLOCKED
        opts.fp64_products = fp64_products
        return H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(),
                                   opts=opts, check=check)
    return call


def _variant(H, code, m, n):
    def call(dA, dB, check):
        return H.hsma_trsm(code, H.RIGHT, H.UPPER, H.TRANS, 0, m, n, 1.0, dA.data_ptr(), n, dB.data_ptr(), m,
                           H.stream_ptr(), check=check)
    return call


CASES = {
    "blocked_fp64": (I.R64, 300, 40, lambda H: _blocked(H, I.R64, 300, 40), None),
    "blocked_c128": (I.C128, 200, 30, lambda H: _blocked(H, I.C128, 200, 30), None),
    "emulated_fp64": (I.R64, 700, 20, lambda H: _blocked(H, I.R64, 700, 20, 1), None),
    "right_upper_trans": (I.R64, 50, 90, lambda H: _variant(H, I.R64, 50, 90), "right"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_alloc_failure_reported_and_recovered(H, name, monkeypatch):
    import torch
    code, m, n, make, kind = CASES[name]
    na = n if kind == "right" else m
    L = I.gen_A(7, na, code)
    A = np.asfortranarray(L.T.copy()) if kind == "right" else L
    B = I.gen_B(7, m, n, code)
    dA, dB = H.to_device(A), H.to_device(B)
    call = make(H)
    monkeypatch.setenv("HSMA_FAULT_ALLOC_AFTER", "0")
    assert call(dA, dB, False) == H.ERR_NO_MEMORY
    torch.cuda.synchronize()
    assert np.array_equal(H.from_device(dB), B), "B written although the call failed"
    monkeypatch.delenv("HSMA_FAULT_ALLOC_AFTER")
    assert call(dA, dB, False) == H.OK
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0
    X = H.from_device(dB)
    ref = oracle.solve_general(A, B, 1.0, 1, 1, 1, False) if kind == "right" else oracle.solve(A, B, 1.0)
    assert oracle.forward_error(X, ref) <= 1e-12


def test_batched_alloc_failure(H, monkeypatch):
    import torch
    ms, ns = I.batched_sizes(6, 200)
    As = [I.gen_A(6, int(m), I.R64, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(6, int(m), int(n), I.R64, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    bt = U.Batch(As, Bs)
    before = bt.dB.clone()
    a = bt.args()
    monkeypatch.setenv("HSMA_FAULT_ALLOC_AFTER", "0")
    s = H.hsma_trsm_llnn_vbatched(I.R64, 0, bt.batch, a[0], a[1], 1.0, a[2], a[3], a[4], a[5], max_m=64,
                                  stream=H.stream_ptr(), check=False)
    assert s == H.ERR_NO_MEMORY
    torch.cuda.synchronize()
    assert torch.equal(bt.dB, before)
    # the allocation-free entry point does not allocate, so the injection does not reach it
    s = H.hsma_trsm_llnn_vbatched_noalloc(I.R64, 0, bt.batch, a[0], a[1], 1.0, a[2], a[3], a[4], a[5], max_m=64,
                                          d_status=bt.d_status.data_ptr(), stream=H.stream_ptr(), check=False)
    assert s == H.OK
    torch.cuda.synchronize()
    assert bt.status() == 0
    out = bt.results()
    for b in range(0, len(As), 17):
        assert oracle.forward_error(out[b], oracle.solve(As[b], Bs[b], 1.0)) <= 1e-13, b
    monkeypatch.delenv("HSMA_FAULT_ALLOC_AFTER")


def test_host_batch_alloc_failure(H, monkeypatch):
    import torch
    ms, ns = I.batched_sizes(8, 100)
    As = [I.gen_A(8, int(m), I.R64, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(8, int(m), int(n), I.R64, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)[:-1]]).astype(np.int64)
    offB = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]]).astype(np.int64)
    hA = np.concatenate([a.ravel(order="F") for a in As])
    hB = np.concatenate([b.ravel(order="F") for b in Bs])
    hX = np.full_like(hB, 7.0)
    m32, n32 = ms.astype(np.int32), ns.astype(np.int32)
    monkeypatch.setenv("HSMA_FAULT_ALLOC_AFTER", "0")
    s = H.hsma_trsm_llnn_vbatched_host(I.R64, 0, len(As), m32, n32, 1.0, hA.ctypes.data, offA, hB.ctypes.data,
                                       offB, hX.ctypes.data, stream=H.stream_ptr(), check=False)
    assert s == H.ERR_NO_MEMORY
    torch.cuda.synchronize()
    assert np.all(hX == 7.0)
    monkeypatch.delenv("HSMA_FAULT_ALLOC_AFTER")
    H.hsma_trsm_llnn_vbatched_host(I.R64, 0, len(As), m32, n32, 1.0, hA.ctypes.data, offA, hB.ctypes.data, offB,
                                   hX.ctypes.data, stream=H.stream_ptr())
    torch.cuda.synchronize()
    for b in range(len(As)):
        got = hX[offB[b]:offB[b] + ms[b] * ns[b]].reshape((ms[b], ns[b]), order="F")
        assert oracle.forward_error(got, oracle.solve(As[b], Bs[b], 1.0)) <= 1e-13, b
