"""The library's kernel-launch counter (hsma_trace_launches) counts every kernel a call
launches, including phases that run several kernels and excluding copies: the figure
bench.py reports as gpu_launches."""
import numpy as np
import pytest

from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _mix(code, batch, seed):
    ms, ns = I.batched_sizes(seed, batch)
    As = [np.asfortranarray(I.gen_A(seed, int(m), code, inst=b)) for b, m in enumerate(ms)]
    Bs = [I.gen_B(seed, int(m), int(n), code, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    return As, Bs


def _count(H, fn):
    import torch
    torch.cuda.synchronize()
    before = H.hsma_trace_launches()
    fn()
    torch.cuda.synchronize()
    return H.hsma_trace_launches() - before


@pytest.mark.parametrize("code,kernels", [(I.C128, 4), (I.R64, 2)])
def test_batch_call_counts_its_kernels(H, code, kernels):
    """complex128: count, place, prep and solve of the column-packed batch; FP64: the
    schedule pre-pass and the per-instance solve."""
    As, Bs = _mix(code, 300, 70)
    bt = U.Batch(As, Bs)
    a = bt.args()
    n = _count(H, lambda: H.hsma_trsm_llnn_vbatched(code, 0, bt.batch, a[0], a[1], 1.0, a[2], a[3], a[4], a[5],
                                                    max_m=64, max_n=0, d_status=bt.d_status.data_ptr(),
                                                    stream=H.stream_ptr()))
    assert n == kernels


def test_factor_solve_batches_count_their_kernels(H):
    """complex128 LU-factor solves: the row-interchange pass, then two packed batches of
    four kernels; without pivots, and for Cholesky factors, the two batches alone."""
    import torch
    As, Bs = _mix(I.C128, 200, 71)
    bt = U.Batch(As, Bs)
    a = bt.args()
    piv = torch.from_numpy(np.concatenate([np.arange(1, A.shape[0] + 1, dtype=np.int32) for A in As])).cuda()
    off = np.concatenate([[0], np.cumsum([A.shape[0] for A in As])[:-1]]).astype(np.int64)
    dptr = torch.from_numpy((piv.data_ptr() + 4 * off).astype(np.int64)).cuda()
    st = H.stream_ptr()
    getrs = lambda p: H.hsma_getrs_vbatched(I.C128, bt.batch, a[0], a[1], 1.0, a[2], a[3], p, a[4], a[5], 64, 64,
                                            bt.d_status.data_ptr(), st)
    assert _count(H, lambda: getrs(dptr.data_ptr())) == 9
    assert _count(H, lambda: getrs(0)) == 8
    assert _count(H, lambda: H.hsma_potrs_vbatched(I.C128, bt.batch, a[0], a[1], 1.0, a[2], a[3], a[4], a[5], 64,
                                                   64, bt.d_status.data_ptr(), st)) == 8
    assert bt.status() == 0
