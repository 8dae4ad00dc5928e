"""The autotuned configuration table (Section 4.3.2) on the GPU: the planner's choice
(the nearest table entry) is at least as fast as a fixed N_B = 256 with the default rest,
within timing noise, and the emulated-products plan reports the table's panel width."""
import pytest

from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _best_ms(H, code, m, n, opts, reps=5):
    import torch
    dt = torch.complex128 if code == I.C128 else torch.float64
    A = torch.empty((m, m), dtype=dt, device="cuda")
    B0 = torch.empty((n, m), dtype=dt, device="cuda")
    H.hsma_gen_matrix(code, 0, 3, -1, m, m, A.data_ptr(), m, H.stream_ptr())
    H.hsma_gen_matrix(code, 1, 3, -1, m, n, B0.data_ptr(), m, H.stream_ptr())
    B = B0.clone()
    best = float("inf")
    for k in range(reps + 1):
        B.copy_(B0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, A.data_ptr(), m, B.data_ptr(), m, H.stream_ptr(), opts=opts)
        e1.record()
        torch.cuda.synchronize()
        if k:
            best = min(best, e0.elapsed_time(e1))
    return best


@pytest.mark.parametrize("code,m,n", [(I.R64, 2048, 256), (I.R64, 8192, 16), (I.C128, 2048, 2048),
                                      (I.C128, 512, 256)])
def test_table_choice_at_least_as_fast_as_fixed_nb(H, code, m, n):
    table = _best_ms(H, code, m, n, H.Opts())
    fixed = H.Opts()
    fixed.nb = 256
    fixed.tile, fixed.split_k, fixed.looking = 0, 1, 1
    ref = _best_ms(H, code, m, n, fixed)
    p = H.hsma_plan(code, m, n)
    assert table <= 1.10 * ref, (p.nb, p.tile, p.split_k, p.looking, table, ref)


def test_emulated_plan_reports_table_panel(H):
    import torch
    m = n = 4096
    o = H.Opts()
    o.fp64_products = 1
    info = H.Info()
    A = torch.empty((m, m), dtype=torch.float64, device="cuda")
    B = torch.empty((n, m), dtype=torch.float64, device="cuda")
    H.hsma_gen_matrix(I.R64, 0, 1, -1, m, m, A.data_ptr(), m, H.stream_ptr())
    H.hsma_gen_matrix(I.R64, 1, 1, -1, m, n, B.data_ptr(), m, H.stream_ptr())
    H.hsma_trsm_llnn_ex(I.R64, 0, m, n, 1.0, A.data_ptr(), m, B.data_ptr(), m, H.stream_ptr(), opts=o, info=info)
    torch.cuda.synchronize()
    assert info.plan.nb in (256, 512) and info.plan.panel_cols in (1024, 2048, 3072, 4096)
