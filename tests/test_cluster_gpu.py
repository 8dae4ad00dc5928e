"""The tensor-core product without clusters (HSMA_TC_CLUSTER=1, read once per
process, so the check runs in a child process): the emulated FP64 product is
still exact on integer data and the emulated blocked solve still matches the
oracle, with an odd number of row tiles (a cluster partner would be missing)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U
H = U.lib()
rng = np.random.default_rng(5)
for M, N, K in ((300, 200, 77), (129, 257, 1024), (1000, 513, 1000)):
    A = np.asfortranarray(rng.integers(-1024, 1025, (M, K)).astype(np.float64))
    X = np.asfortranarray(rng.integers(-1024, 1025, (K, N)).astype(np.float64))
    C0 = np.asfortranarray(rng.integers(-2 ** 20, 2 ** 20, (M, N)).astype(np.float64))
    dA, dX, dC = H.to_device(A), H.to_device(X), H.to_device(C0)
    H.hsma_gemm_f64_emulated(M, N, K, dA.data_ptr(), M, dX.data_ptr(), K, dC.data_ptr(), M, H.stream_ptr())
    torch.cuda.synchronize()
    exact = C0 - (A.astype(np.int64) @ X.astype(np.int64)).astype(np.float64)
    assert np.array_equal(H.from_device(dC), exact), (M, N, K)
for code, m, n in ((I.R64, 700, 50), (I.C128, 300, 33)):
    A0, B0 = I.gen_A(m, m, code), I.gen_B(m, m, n, code)
    dA, dB = H.to_device(A0), H.to_device(B0)
    o = H.Opts(); o.path = H.PATH_BLOCKED; o.fp64_products = 1
    H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=o)
    torch.cuda.synchronize()
    err = oracle.forward_error(H.from_device(dB), oracle.solve(A0, B0, 1.0))
    assert err <= 1e-12, (code, m, err)
assert H.hsma_device_status() == 0
print("CLUSTER1_OK")
"""


def test_products_without_clusters():
    env = dict(os.environ, HSMA_TC_CLUSTER="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "CLUSTER1_OK" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
