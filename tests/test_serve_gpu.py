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
        # each request's arithmetic does not depend on its neighbours: bit for bit
        assert np.array_equal(X, _alone(H, code, A, B, alpha))
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


def _factor_case(code, m, seed, inst, kind, rng):
    """Inputs of one factor-solve request: packed LU factors with a seeded pivot
    sequence (GETRS), or a lower Cholesky factor (POTRS)."""
    if kind == 1:  # GETRS
        F = I.gen_LU(seed, m, code, inst=inst)
        piv = np.array([int(rng.integers(k, m)) + 1 for k in range(m)], dtype=np.int32)
        return F, piv
    return I.gen_A(seed, m, code, inst=inst), None


def _factor_alone(H, code, kind, F, piv, B, alpha, opts=None):
    """The same factor solve through the entry point the server uses for its size."""
    import torch
    m, n = B.shape
    dF, dB = H.to_device(F), H.to_device(B)
    dP = torch.from_numpy(piv).cuda() if piv is not None else None
    if m <= 64:
        bt = U.Batch([F], [B])
        ptrs = [0]
        if dP is not None:
            pp = torch.tensor([dP.data_ptr()], dtype=torch.int64, device="cuda")
            ptrs = [pp]
        if kind == 1:
            H.hsma_getrs_vbatched(code, 1, bt.d_m.data_ptr(), bt.d_n.data_ptr(), alpha, bt.d_ptrA.data_ptr(),
                                  bt.d_lda.data_ptr(), ptrs[0].data_ptr() if dP is not None else 0,
                                  bt.d_ptrB.data_ptr(), bt.d_ldb.data_ptr(), 64, 64, 0, H.stream_ptr())
        else:
            H.hsma_potrs_vbatched(code, 1, bt.d_m.data_ptr(), bt.d_n.data_ptr(), alpha, bt.d_ptrA.data_ptr(),
                                  bt.d_lda.data_ptr(), bt.d_ptrB.data_ptr(), bt.d_ldb.data_ptr(), 64, 64, 0,
                                  H.stream_ptr())
        torch.cuda.synchronize()
        return bt.results()[0]
    if kind == 1:
        H.hsma_getrs(code, m, n, alpha, dF.data_ptr(), m, dP.data_ptr() if dP is not None else 0, dB.data_ptr(), m,
                     H.stream_ptr(), opts)
    else:
        H.hsma_potrs(code, m, n, alpha, dF.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts)
    torch.cuda.synchronize()
    return H.from_device(dB)


@pytest.mark.parametrize("flags", [0, 2], ids=["dmma", "emulated"])
def test_served_factor_solves_mixed_with_triangular(H, flags):
    """A stream mixing triangular solves with LU-factor (with pivots) and Cholesky-factor
    solves, small (batched, fused factor-solve kernel) and large (blocked path): every
    served result equals the same call alone bit for bit and the oracle's getrs / potrs /
    solve within 1e-12."""
    rng = np.random.default_rng(3)
    t, ms, ns, dts = I.serving_requests(21, 90, m_range=(8, 700), n_range=(1, 80))
    s = H.hsma_server_create(1 << 30, 4, flags)
    keep = []
    for k in range(len(ms)):
        code, m, n = int(dts[k]), int(ms[k]), int(ns[k])
        kind = k % 3
        alpha = 1.25 if code == I.R64 else 0.5 + 1.5j
        B = I.gen_B(21, m, n, code, inst=k)
        if kind == 0:
            F, piv = I.gen_A(21, m, code, inst=k), None
        else:
            F, piv = _factor_case(code, m, 21, k, kind, rng)
        X = np.zeros_like(B, order="F")
        r = H.Request()
        r.dtype, r.diag, r.m, r.n, r.kind = code, 0, m, n, kind
        r.alpha[0], r.alpha[1] = complex(alpha).real, complex(alpha).imag
        r.A_host, r.lda, r.B_host, r.ldb = F.ctypes.data, m, B.ctypes.data, m
        r.X_host, r.ldx = X.ctypes.data, m
        if piv is not None:
            r.ipiv_host = piv.ctypes.data
        keep.append((code, kind, F, piv, B, X, alpha, r, H.hsma_server_submit(s, r)))
    assert H.hsma_server_drain(s, 180.0) == 0
    st = H.hsma_server_stats(s)
    assert st.completed == len(ms) and st.batched_launches >= 3 and st.blocked_launches >= 3
    for code, kind, F, piv, B, X, alpha, _, tk in keep:
        assert H.hsma_server_poll(s, tk)[2] == 0
        m, n = B.shape
        opts = H.Opts()
        opts.fp64_products = 1 if (flags and m >= 384) else 0
        if kind == 0:
            import torch
            dA, dB = H.to_device(F), H.to_device(B)
            H.hsma_trsm_llnn_ex(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts)
            torch.cuda.synchronize()
            alone = H.from_device(dB)
            ref = oracle.solve(F, B, alpha)
        else:
            alone = _factor_alone(H, code, kind, F, piv, B, alpha, opts)
            ref = oracle.getrs(F, piv, B, alpha) if kind == 1 else oracle.potrs(F, B, alpha)
        assert np.array_equal(X, alone), (kind, m, n)
        assert oracle.forward_error(X, ref) <= 1e-12, (kind, m, n)
    assert H.hsma_device_status() == 0
    assert H.hsma_server_destroy(s) == 0


def test_served_generated_factor_inputs(H):
    """Factor-solve requests with device-generated inputs: packed LU factors (generator
    kind 2, no interchanges) and Cholesky factors (kind 0) match the host generator."""
    s = H.hsma_server_create(1 << 30, 2, 0)
    cases = [(I.R64, 40, 7, 1), (I.C128, 200, 9, 1), (I.C128, 30, 3, 2), (I.R64, 150, 20, 2)]
    outs = []
    for k, (code, m, n, kind) in enumerate(cases):
        X = np.zeros((m, n), dtype=np.float64 if code == I.R64 else np.complex128, order="F")
        r = H.Request()
        r.dtype, r.diag, r.m, r.n, r.kind = code, 0, m, n, kind
        r.alpha[0], r.alpha[1] = 1.0, 0.0
        r.gen_seed, r.gen_inst = 91, k
        r.X_host, r.ldx = X.ctypes.data, m
        outs.append((code, m, n, kind, k, X, r))
        H.hsma_server_submit(s, r)
    assert H.hsma_server_drain(s, 60.0) == 0
    for code, m, n, kind, k, X, _ in outs:
        B = I.gen_B(91, m, n, code, inst=k)
        if kind == 1:
            ref = oracle.getrs(I.gen_LU(91, m, code, inst=k), None, B, 1.0)
        else:
            ref = oracle.potrs(I.gen_A(91, m, code, inst=k), B, 1.0)
        assert oracle.forward_error(X, ref) <= 1e-12, (kind, m, n)
    assert H.hsma_server_destroy(s) == 0


def test_serving_stream_at_workload_scale(H):
    """The serving workload's size mix (m log-uniform in [16, 4096], n in [1, 512], 30%
    complex128) at its arrival rate, submitted from a second thread while earlier
    requests run; device-generated inputs; every request completes within a 4 GB budget,
    and a seeded sample is checked against the oracle and against the same request
    solved alone (bit for bit)."""
    import threading
    import time
    import torch
    count = 500
    t_arr, ms, ns, dts = I.serving_requests(44, count)
    budget = 4 << 30
    s = H.hsma_server_create(budget, 8, 0)
    sample = set(np.random.default_rng(44).choice(count, 6, replace=False).tolist())
    outs, reqs, tickets = {}, [], [None] * count
    for k in range(count):
        r = H.Request()
        r.dtype, r.diag, r.m, r.n = int(dts[k]), 0, int(ms[k]), int(ns[k])
        r.alpha[0], r.alpha[1] = 1.0, 0.0
        r.gen_seed, r.gen_inst = 44, k
        if k in sample:
            X = np.zeros((int(ms[k]), int(ns[k])), dtype=np.float64 if dts[k] == I.R64 else np.complex128,
                         order="F")
            r.X_host, r.ldx = X.ctypes.data, int(ms[k])
            outs[k] = X
        reqs.append(r)

    def producer():
        t0 = time.perf_counter()
        for k in range(count):
            while time.perf_counter() - t0 < t_arr[k]:
                time.sleep(0.0002)
            tickets[k] = H.hsma_server_submit(s, reqs[k])

    th = threading.Thread(target=producer)
    th.start()
    overlap = 0
    while th.is_alive():  # the main thread watches completions while arrivals continue
        st = H.hsma_server_stats(s)
        overlap = max(overlap, st.submitted - st.completed)
        time.sleep(0.002)
    th.join()
    assert H.hsma_server_drain(s, 120.0) == 0
    st = H.hsma_server_stats(s)
    assert st.completed == count and st.peak_bytes_in_use <= budget
    assert overlap >= 2  # requests were in flight while others arrived
    for k in range(count):
        assert H.hsma_server_poll(s, tickets[k])[2] == 0
    for k, X in outs.items():
        code, m, n = int(dts[k]), int(ms[k]), int(ns[k])
        dt = torch.complex128 if code == I.C128 else torch.float64
        dA = torch.empty((m, m), dtype=dt, device="cuda")
        dB = torch.empty((n, m), dtype=dt, device="cuda")
        H.hsma_gen_matrix(code, 0, 44, k, m, m, dA.data_ptr(), m, H.stream_ptr())
        H.hsma_gen_matrix(code, 1, 44, k, m, n, dB.data_ptr(), m, H.stream_ptr())
        torch.cuda.synchronize()
        A, B = np.asfortranarray(dA.cpu().numpy().T), np.asfortranarray(dB.cpu().numpy().T)
        H.hsma_trsm_llnn(code, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(X, np.asfortranarray(dB.cpu().numpy().T)), (k, m, n)
        assert oracle.forward_error(X, oracle.solve(A, B, 1.0)) <= 1e-12, (k, m, n)
    assert H.hsma_server_destroy(s) == 0
