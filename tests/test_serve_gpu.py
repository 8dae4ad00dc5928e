"""Serving loop on the GPU: every result served in the mix equals the request
solved alone and the oracle (within 1e-12); the memory budget holds."""
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


def _alone(H, code, A, B, alpha):
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    m, n = B.shape
    H.hsma_trsm_llnn(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
    torch.cuda.synchronize()
    return H.from_device(dB)


def test_served_results_equal_alone_and_oracle(H):
    t, ms, ns, dts = I.serving_requests(5, 160, m_range=(16, 700), n_range=(1, 96))
    keep, reqs, tickets = [], [], []
    budget = 256 << 20
    s = H.hsma_server_create(budget, 4, 0)
    for k in range(len(ms)):
        code = int(dts[k])
        m, n = int(ms[k]), int(ns[k])
        A, B = I.gen_A(5, m, code, inst=k), I.gen_B(5, m, n, code, inst=k)
        X = np.zeros_like(B, order="F")
        alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
        r = H.Request()
        r.dtype, r.diag, r.m, r.n = code, 0, m, n
        r.alpha[0], r.alpha[1] = complex(alpha).real, complex(alpha).imag
        r.A_host, r.lda, r.B_host, r.ldb = A.ctypes.data, m, B.ctypes.data, m
        r.X_host, r.ldx = X.ctypes.data, m
        keep.append((code, A, B, X, alpha))
        reqs.append(r)
        tickets.append(H.hsma_server_submit(s, r))
    assert H.hsma_server_drain(s, 120.0) == 0
    st = H.hsma_server_stats(s)
    assert st.completed == len(ms) and st.peak_bytes_in_use <= budget
    assert st.batched_launches >= 1 and st.blocked_launches >= 1
    for tk, (code, A, B, X, alpha) in zip(tickets, keep):
        done, lat, status = H.hsma_server_poll(s, tk)
        assert done and status == 0 and lat > 0
        ref = oracle.solve(A, B, alpha)
        assert oracle.forward_error(X, ref) <= 1e-12
        assert oracle.forward_error(X, _alone(H, code, A, B, alpha)) <= 1e-12
    assert H.hsma_server_destroy(s) == 0


def test_served_device_generated_inputs(H):
    """Requests whose A and B are generated on the device from (seed, instance)."""
    s = H.hsma_server_create(1 << 30, 3, 0)
    cases = [(I.R64, 37, 5), (I.C128, 100, 17), (I.R64, 300, 1), (I.C128, 64, 64)]
    outs = []
    for k, (code, m, n) in enumerate(cases):
        X = np.zeros((m, n), dtype=np.float64 if code == I.R64 else np.complex128, order="F")
        r = H.Request()
        r.dtype, r.diag, r.m, r.n = code, 0, m, n
        r.alpha[0], r.alpha[1] = 1.0, 0.0
        r.gen_seed, r.gen_inst = 77, k
        r.X_host, r.ldx = X.ctypes.data, m
        outs.append((code, m, n, k, X, r))
        H.hsma_server_submit(s, r)
    assert H.hsma_server_drain(s, 60.0) == 0
    for code, m, n, k, X, _ in outs:
        A, B = I.gen_A(77, m, code, inst=k), I.gen_B(77, m, n, code, inst=k)
        assert oracle.forward_error(X, oracle.solve(A, B, 1.0)) <= 1e-12
    assert H.hsma_server_destroy(s) == 0


def test_served_emulated_results_equal_alone_and_oracle(H):
    """HSMA_SERVER_FP64_EMULATED: requests with m >= 384 use the emulated FP64 products; each result
    is bitwise the same request solved alone with the same products, and within 1e-12 of the oracle."""
    import torch
    t, ms, ns, dts = I.serving_requests(8, 24, m_range=(65, 900), n_range=(1, 96))
    s = H.hsma_server_create(1 << 30, 4, H.SERVER_FP64_EMULATED)
    keep = []
    for k in range(len(ms)):
        code, m, n = int(dts[k]), int(ms[k]), int(ns[k])
        A, B = I.gen_A(8, m, code, inst=k), I.gen_B(8, m, n, code, inst=k)
        X = np.zeros_like(B, order="F")
        alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
        r = H.Request()
        r.dtype, r.diag, r.m, r.n = code, 0, m, n
        r.alpha[0], r.alpha[1] = complex(alpha).real, complex(alpha).imag
        r.A_host, r.lda, r.B_host, r.ldb = A.ctypes.data, m, B.ctypes.data, m
        r.X_host, r.ldx = X.ctypes.data, m
        keep.append((code, A, B, X, alpha, r, H.hsma_server_submit(s, r)))
    assert H.hsma_server_drain(s, 120.0) == 0
    assert H.hsma_server_stats(s).blocked_launches >= 1
    for code, A, B, X, alpha, _, tk in keep:
        assert H.hsma_server_poll(s, tk)[2] == 0
        dA, dB = H.to_device(A), H.to_device(B)
        m, n = B.shape
        opts = H.Opts()
        opts.fp64_products = 1 if m >= 384 else 0  # the server's rule
        H.hsma_trsm_llnn_ex(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts)
        torch.cuda.synchronize()
        assert np.array_equal(X, H.from_device(dB))
        assert oracle.forward_error(X, oracle.solve(A, B, alpha)) <= 1e-12
    assert H.hsma_server_destroy(s) == 0
