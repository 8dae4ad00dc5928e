"""Reduced-precision modes: the BF16 tensor-core update (tcgen05), the FP32-result
solve (<= 2e-5 against the FP64 oracle of the FP64 data) and the FP64-result
solve by iterative refinement (<= 1e-12)."""
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


def _bf16_values(rng, shape):
    """float32 values exactly representable in BF16 (8-bit significands)."""
    mant = rng.integers(-128, 128, shape).astype(np.float32)
    expo = rng.integers(-6, 2, shape).astype(np.float32)
    return (mant * np.exp2(expo - 7)).astype(np.float32)


def _bf16_bits(x32):
    return (x32.view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("M,N,K,beta", [(300, 600, 192, 1.0), (128, 256, 64, 0.5), (77, 5, 128, 1.0),
                                        (1000, 513, 768, 1.0), (2100, 2600, 128, 1.0), (4000, 5000, 64, 0.5)])
def test_bf16_update_parity(H, M, N, K, beta):
    import torch
    rng = np.random.default_rng(M + N + K)
    A = _bf16_values(rng, (M, K))
    Bt = _bf16_values(rng, (N, K))
    C0 = rng.uniform(-1, 1, (M, N)).astype(np.float32)
    ldc = M + 3
    Cb = np.full((ldc, N), 5.0, dtype=np.float32, order="F")
    Cb[:M] = C0
    dA = torch.from_numpy(_bf16_bits(A)).cuda()       # row-major M x K
    dB = torch.from_numpy(_bf16_bits(Bt)).cuda()      # row-major N x K
    dC = H.to_device(Cb)
    H.hsma_gemm_bf16_update(M, N, K, dA.data_ptr(), dB.data_ptr(), beta, dC.data_ptr(), ldc, H.stream_ptr())
    torch.cuda.synchronize()
    got = H.from_device(dC)
    ref = beta * C0.astype(np.float64) - A.astype(np.float64) @ Bt.astype(np.float64).T
    scale = np.abs(C0) + np.abs(A.astype(np.float64)) @ np.abs(Bt.astype(np.float64)).T
    assert np.all(np.abs(got[:M] - ref) <= 1e-5 * scale + 1e-30), np.max(np.abs(got[:M] - ref) / scale)
    assert np.all(got[M:] == 5.0)
    assert H.hsma_device_status() == 0


def _r32(H, A64, B64, alpha, terms=0, nb=0):
    import torch
    A32 = np.asfortranarray(A64.astype(np.float32))
    B32 = np.asfortranarray(B64.astype(np.float32))
    dA, dB = H.to_device(A32), H.to_device(B32)
    opts = H.Opts()
    opts.bf16_terms = terms
    opts.nb = nb
    m, n = B64.shape
    H.hsma_trsm_llnn_ex(H.R32_BF16, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    return H.from_device(dB).astype(np.float64)


@pytest.mark.parametrize("m,n,nb", [(1000, 300, 128), (517, 77, 64), (64, 64, 64), (2048, 100, 256),
                                     (1500, 37, 512), (777, 50, 256), (4096, 20, 512)])
def test_r32_mode_accuracy(H, m, n, nb):
    A, B = I.gen_A(7, m, I.R64), I.gen_B(7, m, n, I.R64)
    X = _r32(H, A, B, 1.5, terms=3, nb=nb)
    err = oracle.forward_error(X, oracle.solve(A, B, 1.5))
    assert err <= 2e-5, err
    assert H.hsma_device_status() == 0


def test_r32_mode_config3_sampled(H):
    """m = 8192, n = 4096 FP32-result mode, split BF16 (3 terms), sampled columns."""
    import torch
    m, n = 8192, 4096
    A = I.gen_A(0, m, I.R64)
    B = I.gen_B(0, m, n, I.R64)
    X = _r32(H, A, B, 1.0)
    cols = np.arange(0, n, 64)
    ref = oracle.solve_cols(A, B, 1.0, cols)
    err = oracle.forward_error(X[:, cols], ref)
    assert err <= 2e-5, err


def _ir(H, A, B, alpha, **kw):
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    opts = H.Opts()
    for k, v in kw.items():
        setattr(opts, k, v)
    info = H.Info()
    m, n = B.shape
    H.hsma_trsm_llnn_ex(H.R64_IR, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts,
                        info=info)
    torch.cuda.synchronize()
    return H.from_device(dB), info


@pytest.mark.parametrize("residual", [0, 1], ids=["emulated", "dmma"])
@pytest.mark.parametrize("m,n", [(1000, 300), (300, 1000), (129, 1), (2000, 64)])
def test_ir_mode_reaches_fp64_accuracy(H, m, n, residual):
    """FP64-result mode; residual products emulated on the BF16 tensor cores (exact
    integer slices) or FP64 tensor products."""
    A, B = I.gen_A(9, m, I.R64), I.gen_B(9, m, n, I.R64)
    X, info = _ir(H, A, B, 1.5, ir_residual=residual)
    assert info.converged == 1 and 1 <= info.ir_iters <= 10
    assert info.ir_residual <= 1e-15
    err = oracle.forward_error(X, oracle.solve(A, B, 1.5))
    assert err <= 1e-12, err
    assert oracle.backward_error(A, B, X, 1.5) <= 1e-14
    assert H.hsma_device_status() == 0


def test_ir_mode_unit_diagonal_emulated(H):
    m, n = 700, 90
    A0, B = I.gen_A(12, m, I.R64), I.gen_B(12, m, n, I.R64)
    A = np.array(A0, order="F")
    np.fill_diagonal(A, np.nan)  # never read under a unit diagonal
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    info = H.Info()
    H.hsma_trsm_llnn_ex(H.R64_IR, 1, m, n, -0.5, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=H.Opts(),
                        info=info)
    torch.cuda.synchronize()
    A1 = np.array(A0, order="F")
    np.fill_diagonal(A1, 1.0)
    X = H.from_device(dB)
    assert info.converged == 1
    assert oracle.forward_error(X, oracle.solve(A1, B, -0.5)) <= 1e-12


def test_ir_not_converged_reported_without_info(H):
    """A refinement that cannot reach its tolerance within ir_max_iter steps is not
    silent: called with no info block the solve returns OK (asynchronous) but the
    device error word carries HSMA_DEVERR_NOT_CONVERGED; with an info block the
    call returns HSMA_ERR_NOT_CONVERGED."""
    import torch
    m, n = 600, 40
    A, B = I.gen_A(21, m, I.R64), I.gen_B(21, m, n, I.R64)
    assert H.hsma_device_status() == 0
    opts = H.Opts()
    opts.ir_max_iter = 1
    opts.ir_tol = 1e-300  # unreachable
    dA, dB = H.to_device(A), H.to_device(B)
    s = H.hsma_trsm_llnn_ex(H.R64_IR, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts)
    assert s == 0
    torch.cuda.synchronize()
    assert H.hsma_device_status() == H.DEVERR_NOT_CONVERGED
    assert H.hsma_device_status() == 0  # cleared by the read
    # the result is still the refined one (one step), within the FP64 tolerance
    assert oracle.forward_error(H.from_device(dB), oracle.solve(A, B, 1.0)) <= 1e-12
    dB = H.to_device(B)
    info = H.Info()
    s = H.hsma_trsm_llnn_ex(H.R64_IR, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts,
                            info=info, check=False)
    torch.cuda.synchronize()
    assert s == 6 and info.converged == 0 and info.ir_iters == 1
    H.hsma_device_status()
    # a reachable tolerance raises nothing
    dB = H.to_device(B)
    H.hsma_trsm_llnn_ex(H.R64_IR, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
    torch.cuda.synchronize()
    assert H.hsma_device_status() == 0


def test_ir_mode_config3_sampled(H):
    """FP64-result mode at the m = 8192, n = 4096 workload size: forward error on 64
    sampled columns against the FP64 oracle (exact per column) <= 1e-12, and the
    normwise residual ratio reported by the refinement <= 1e-15."""
    m, n = 8192, 4096
    A = I.gen_A(0, m, I.R64)
    B = I.gen_B(0, m, n, I.R64)
    X, info = _ir(H, A, B, 1.0)
    assert info.converged == 1 and info.ir_residual <= 1e-15
    cols = np.arange(0, n, 64)
    ref = oracle.solve_cols(A, B, 1.0, cols)
    err = oracle.forward_error(X[:, cols], ref)
    assert err <= 1e-12, err
    assert H.hsma_device_status() == 0


def test_workspace_pool_does_not_grow(H):
    """Workspace comes from the library's stream-ordered pool: after the first call,
    repeated FP32-result and refinement solves with a synchronisation between them
    take no further device memory (released workspace is reused, nothing leaks)."""
    import torch
    m, n = 1536, 200
    A64, B64 = I.gen_A(9, m, I.R64), I.gen_B(9, m, n, I.R64)
    A32 = torch.from_numpy(np.ascontiguousarray(A64.T)).float().cuda()
    B32 = torch.from_numpy(np.ascontiguousarray(B64.T)).float().cuda()
    A = torch.from_numpy(np.ascontiguousarray(A64.T)).cuda()
    B0 = torch.from_numpy(np.ascontiguousarray(B64.T)).cuda()
    X32, X = B32.clone(), B0.clone()

    def solve_both():
        X32.copy_(B32)
        X.copy_(B0)
        H.hsma_trsm_llnn_ex(H.R32_BF16, 0, m, n, 1.0, A32.data_ptr(), m, X32.data_ptr(), m, H.stream_ptr())
        H.hsma_trsm_llnn_ex(H.R64_IR, 0, m, n, 1.0, A.data_ptr(), m, X.data_ptr(), m, H.stream_ptr())
        torch.cuda.synchronize()

    solve_both()
    free_after_first = torch.cuda.mem_get_info()[0]
    for _ in range(8):
        solve_both()
    assert torch.cuda.mem_get_info()[0] >= free_after_first - (64 << 20)
    assert oracle.forward_error(X.cpu().numpy().T, oracle.solve(A64, B64, 1.0)) <= 1e-12
