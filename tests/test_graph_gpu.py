"""The varlen batched solve captured into a CUDA graph and replayed."""
import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def test_vbatched_graph_replay_matches_eager():
    import torch
    H = U.lib()
    alpha = 1.5 - 0.5j
    ms, ns = I.batched_sizes(3, 500)
    As = [I.gen_A(3, int(m), I.C128, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(3, int(m), int(n), I.C128, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    eager = U.Batch(As, Bs)
    H.hsma_trsm_llnn_vbatched(I.C128, 0, eager.batch, *eager.args()[:2], alpha, *eager.args()[2:], max_m=64,
                              stream=H.stream_ptr())
    torch.cuda.synchronize()
    ref = eager.results()
    bt = U.Batch(As, Bs)
    B0 = bt.dB.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            H.hsma_trsm_llnn_vbatched(I.C128, 0, bt.batch, *bt.args()[:2], alpha, *bt.args()[2:], max_m=64,
                                      stream=int(s.cuda_stream))
    torch.cuda.synchronize()
    for _ in range(3):  # each replay solves the restored inputs again
        bt.dB.copy_(B0)
        g.replay()
        torch.cuda.synchronize()
        got = bt.results()
        for b in range(bt.batch):
            assert np.array_equal(got[b], ref[b]), b
    refs = oracle.solve_batch(As[:20], Bs[:20], alpha)
    for b in range(20):
        assert oracle.forward_error(got[b], refs[b]) <= 1e-12


def test_getrs_graph_replay_matches_eager():
    """The fused LU-factor solve (with row interchanges) captured into a CUDA graph."""
    import torch
    la = pytest.importorskip("scipy.linalg")
    H = U.lib()
    alpha = 0.5 - 1.0j
    ms, ns = I.batched_sizes(4, 300)
    rng = np.random.default_rng(4)
    LUs, pivs, Bs = [], [], []
    for m, n in zip(ms, ns):
        m, n = int(m), int(n)
        A = (rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) / np.sqrt(m) + 2.0 * np.eye(m)
        lu, piv = la.lu_factor(A[rng.permutation(m)])
        LUs.append(np.asfortranarray(lu))
        pivs.append((piv + 1).astype(np.int32))
        Bs.append(np.asfortranarray(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))))
    off = np.concatenate([[0], np.cumsum([len(p) for p in pivs])[:-1]]).astype(np.int64)
    dpiv = torch.from_numpy(np.concatenate(pivs)).cuda()
    dptr = torch.from_numpy((dpiv.data_ptr() + 4 * off).astype(np.int64)).cuda()

    def call(bt, st):
        a = bt.args()
        H.hsma_getrs_vbatched(I.C128, bt.batch, a[0], a[1], alpha, a[2], a[3], dptr.data_ptr(), a[4], a[5], max_m=64,
                              stream=st)

    eager = U.Batch(LUs, Bs)
    call(eager, H.stream_ptr())
    torch.cuda.synchronize()
    ref = eager.results()
    bt = U.Batch(LUs, Bs)
    B0 = bt.dB.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            call(bt, int(s.cuda_stream))
    torch.cuda.synchronize()
    for _ in range(2):
        bt.dB.copy_(B0)
        g.replay()
        torch.cuda.synchronize()
        got = bt.results()
        for b in range(bt.batch):
            assert np.array_equal(got[b], ref[b]), b
    for b in range(0, bt.batch, 29):
        assert oracle.forward_error(got[b], oracle.getrs(LUs[b], pivs[b], Bs[b], alpha)) <= 1e-12, b


def _capture_solve(H, code, A, B0, alpha, m, n, opts=None, info=None):
    """The single solve on a copy of B0 captured into a CUDA graph; returns (graph, B)."""
    import torch
    B = B0.clone()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            H.hsma_trsm_llnn_ex(code, 0, m, n, alpha, A.data_ptr(), m, B.data_ptr(), m, int(s.cuda_stream),
                                opts=opts, info=info)
    torch.cuda.synchronize()
    return g, B


@pytest.mark.parametrize("m,n,nb", [(1500, 96, 512), (700, 33, 128)])
def test_r32_mode_graph_replay_matches_eager(m, n, nb):
    """The FP32-result solve captured into a CUDA graph: its panel conversion runs on
    the library's side stream (forked and joined by events), its inverses by doubling;
    every replay gives the eager result bit for bit."""
    import torch
    H = U.lib()
    A64, B64 = I.gen_A(5, m, I.R64), I.gen_B(5, m, n, I.R64)
    A = torch.from_numpy(np.ascontiguousarray(A64.T)).float().cuda()  # column-major m x m
    B0 = torch.from_numpy(np.ascontiguousarray(B64.T)).float().cuda()
    opts = H.Opts()
    opts.nb = nb
    eager = B0.clone()
    H.hsma_trsm_llnn_ex(H.R32_BF16, 0, m, n, 1.5, A.data_ptr(), m, eager.data_ptr(), m, H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    g, B = _capture_solve(H, H.R32_BF16, A, B0, 1.5, m, n, opts=opts)
    for _ in range(2):
        B.copy_(B0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(B, eager)
    X = eager.double().cpu().numpy().T
    assert oracle.forward_error(X, oracle.solve(A64.astype(np.float32).astype(np.float64),
                                                B64.astype(np.float32).astype(np.float64), 1.5)) <= 2e-5


def test_ir_mode_graph_replay_matches_eager():
    """The FP64-result refinement captured into a CUDA graph: every refinement step is
    recorded and the device skips those after convergence; a replay gives the eager
    result bit for bit and FP64 accuracy."""
    import torch
    H = U.lib()
    m, n = 900, 40
    A64, B64 = I.gen_A(6, m, I.R64), I.gen_B(6, m, n, I.R64)
    A = torch.from_numpy(np.ascontiguousarray(A64.T)).cuda()
    B0 = torch.from_numpy(np.ascontiguousarray(B64.T)).cuda()
    opts = H.Opts()
    opts.ir_max_iter = 4
    eager = B0.clone()
    H.hsma_trsm_llnn_ex(H.R64_IR, 0, m, n, 1.0, A.data_ptr(), m, eager.data_ptr(), m, H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    g, B = _capture_solve(H, H.R64_IR, A, B0, 1.0, m, n, opts=opts)
    B.copy_(B0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(B, eager)
    X = eager.cpu().numpy().T
    assert oracle.forward_error(X, oracle.solve(A64, B64, 1.0)) <= 1e-12
    assert H.hsma_device_status() == 0
