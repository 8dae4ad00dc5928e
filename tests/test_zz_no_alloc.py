"""The allocation-free batched entry point against the allocating one.

Some callers cannot let the library allocate device memory while solving (a
serving loop that reserved the whole GPU up front, an application whose own
allocator owns all device memory).  hsma_trsm_llnn_vbatched_noalloc keeps the
batch schedule in a static device array instead; it must give the same results
as hsma_trsm_llnn_vbatched, call after call.  This file is collected last.
"""
import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _batch(code, batch, seed):
    ms, ns = I.batched_sizes(seed, batch)
    As = [I.gen_A(seed, int(m), code, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(seed, int(m), int(n), code, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    return As, Bs


@pytest.mark.parametrize("code", [I.C128, I.R64])
def test_noalloc_matches_allocating_entry_point_twice(code):
    import torch
    H = U.lib()
    alpha = 1.5 - 0.5j if code == I.C128 else 1.5
    As, Bs = _batch(code, 3000, seed=17)
    ref_bt = U.Batch(As, Bs)
    H.hsma_trsm_llnn_vbatched(code, 0, ref_bt.batch, *ref_bt.args()[:2], alpha, *ref_bt.args()[2:], max_m=64,
                              max_n=64, d_status=ref_bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    ref = ref_bt.results()
    assert ref_bt.status() == 0
    for call in range(2):  # two calls in a row share the static scratch
        bt = U.Batch(As, Bs)
        H.hsma_trsm_llnn_vbatched_noalloc(code, 0, bt.batch, *bt.args()[:2], alpha, *bt.args()[2:], max_m=64,
                                          max_n=64, d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
        torch.cuda.synchronize()
        assert bt.status() == 0
        got = bt.results()
        for b in range(len(As)):
            assert np.array_equal(got[b], ref[b]), (call, b)
    refs = oracle.solve_batch(As[:50], Bs[:50], alpha)
    for b in range(50):
        assert oracle.forward_error(got[b], refs[b]) <= 1e-12


def test_noalloc_rejects_oversized_batch():
    H = U.lib()
    s = H.hsma_trsm_llnn_vbatched_noalloc(I.R64, 0, 65537, 1, 1, 1.0, 1, 1, 1, 1, check=False)
    assert s == 2  # HSMA_ERR_UNSUPPORTED, nothing launched
