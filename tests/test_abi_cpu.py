"""The C-ABI library loads, exports what include/hsma.h declares, and validates
arguments on the host before touching the GPU (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_2608_25469_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    B.build()
    from paper_2608_25469_gb300 import hsma
    return hsma


def header_functions():
    text = open(os.path.join(ROOT, "include", "hsma.h")).read()
    return sorted(set(re.findall(r"HSMA_API[^;(]*?\b(hsma_\w+)\s*\(", text)))


def test_exports_match_header(H):
    declared = header_functions()
    assert declared, "no declarations found"
    out = os.popen(f"nm -D --defined-only {H.LIB_PATH}").read()
    exported = set(re.findall(r"\bT (hsma_\w+)", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert sorted(H.EXPORTS) == declared, "binding and header disagree"
    for f in declared:
        assert hasattr(H.lib(), f)


def header_arity():
    """Parameter count of every function include/hsma.h declares."""
    text = re.sub(r"/\*.*?\*/|//[^\n]*", "", open(os.path.join(ROOT, "include", "hsma.h")).read(), flags=re.S)
    out = {}
    for name, params in re.findall(r"HSMA_API[^;(]*?\b(hsma_\w+)\s*\(([^;]*?)\)\s*;", text, flags=re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_declares_every_signature(H):
    # without argtypes ctypes passes a Python int as a C int: a 64-bit pointer loses its upper half
    arity = header_arity()
    assert sorted(arity) == header_functions()
    for f, n in arity.items():
        fn = getattr(H.lib(), f)
        if n:
            assert fn.argtypes is not None and len(fn.argtypes) == n, f"{f}: argtypes {fn.argtypes}, header {n}"
        assert fn.restype is not ctypes.c_int or f not in ("hsma_version", "hsma_status_string"), f


def test_version_and_status_strings(H):
    assert re.match(r"\d+\.\d+\.\d+", H.hsma_version())
    for s, name in H.STATUS_NAMES.items():
        assert H.hsma_status_string(s) == name
    assert H.hsma_status_string(999) == "HSMA_ERR_UNKNOWN"


@pytest.mark.parametrize("args", [
    dict(dtype=0, diag=0, m=-1, n=4, lda=4, ldb=4),     # m < 0
    dict(dtype=0, diag=0, m=4, n=-1, lda=4, ldb=4),     # n < 0
    dict(dtype=0, diag=0, m=4, n=4, lda=3, ldb=4),      # lda < m
    dict(dtype=1, diag=0, m=4, n=4, lda=4, ldb=3),      # ldb < m
    dict(dtype=9, diag=0, m=4, n=4, lda=4, ldb=4),      # dtype
    dict(dtype=0, diag=2, m=4, n=4, lda=4, ldb=4),      # diag
    dict(dtype=0, diag=0, m=0, n=4, lda=0, ldb=1),      # lda < max(1, m)
])
def test_invalid_arguments_rejected_without_launch(H, args):
    s = H.hsma_trsm_llnn(args["dtype"], args["diag"], args["m"], args["n"], 1.0, 0, args["lda"], 0, args["ldb"],
                         check=False)
    assert s == 1  # HSMA_ERR_INVALID_ARG


def test_null_pointers_rejected(H):
    assert H.hsma_trsm_llnn(0, 0, 4, 4, 1.0, 0, 4, 0, 4, check=False) == 1


def test_quick_return_empty(H):
    # m == 0 or n == 0: no-op, no pointer is touched, no CUDA call made
    assert H.hsma_trsm_llnn(0, 0, 0, 5, 1.0, 0, 1, 0, 1, check=False) == 0
    assert H.hsma_trsm_llnn(1, 1, 7, 0, 1.0, 0, 7, 0, 7, check=False) == 0
    assert H.hsma_trsm_llnn_vbatched(1, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, check=False) == 0


def test_vbatched_argument_checks(H):
    assert H.hsma_trsm_llnn_vbatched(2, 0, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 2   # dtype unsupported
    assert H.hsma_trsm_llnn_vbatched(7, 0, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 1   # dtype unknown
    assert H.hsma_trsm_llnn_vbatched(0, 0, -1, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 1  # batch < 0
    # max_m > 64 admits large instances (read back from the device): argument errors still come first
    assert H.hsma_trsm_llnn_vbatched(0, 0, 4, 0, 1, 1.0, 1, 1, 1, 1, max_m=65, check=False) == 1
    assert H.hsma_trsm_llnn_vbatched(0, 0, 4, 0, 1, 1.0, 1, 1, 1, 1, check=False) == 1   # NULL d_m


def test_plan_dispatch(H):
    # Section 4.1: 64 is the boundary between the direct solve and the blocked path
    assert H.hsma_plan(H.R64, 64, 64).path == H.PATH_SMALL
    assert H.hsma_plan(H.C128, 64, 4096).path == H.PATH_SMALL
    assert H.hsma_plan(H.R64, 65, 64).path == H.PATH_BLOCKED
    assert H.hsma_plan(H.R32_BF16, 32, 32).path == H.PATH_BLOCKED
    p = H.hsma_plan(H.R64, 16384, 16384)
    assert p.nb in (32, 64, 128, 256, 512)


def test_tuning_table_nearest_match(H, tmp_path):
    # Section 4.3.2: offline table, nearest tested scale at run time
    f = tmp_path / "t.txt"
    f.write_text("# dtype m n nb\n0 100 100 32\n0 2000 2000 64\n0 30000 30000 512\n")
    try:
        assert H.hsma_tuning_load(str(f)) == 0
        assert H.hsma_plan(H.R64, 120, 120).nb == 32
        assert H.hsma_plan(H.R64, 3000, 1500).nb == 64
        assert H.hsma_plan(H.R64, 16384, 16384).nb == 512
        assert H.hsma_plan(H.C128, 120, 120).nb == 32  # no C128 rows: falls back to R64 rows
        bad = tmp_path / "bad.txt"
        bad.write_text("0 100 100 33\n")
        assert H.hsma_tuning_load(str(bad)) == 1
        assert H.hsma_plan(H.R64, 120, 120).nb == 32  # unchanged after a rejected load
    finally:
        assert H.hsma_tuning_load(None) == 0


def test_small_cost_model(H):
    # fp64, G = 1, one tile: R + sum_{i<m-1} (R - (i+1)) with R = m, plus staging
    m = 64
    tile = m + sum(m - (i + 1) for i in range(m - 1))
    stage = sum((m - 1 - i + 31) // 32 for i in range(m))
    assert H.hsma_small_cost(H.R64, m, 32, 1) == tile + stage
    # complex costs four FP64 instructions per multiply-add
    assert H.hsma_small_cost(H.C128, 32, 32, 1) == 4 * H.hsma_small_cost(H.R64, 32, 32, 1)
    assert H.hsma_small_cost(H.C128, 33, 8, 1) == -1.0   # complex G=1 holds 32 rows at most
    assert H.hsma_small_cost(H.R64, 65, 8, 2) == -1.0


def test_vbatched_host_argument_checks(H):
    """The host-buffer batch validates sizes and offsets on the host, before any device call."""
    import numpy as np
    m = np.array([4, 8], dtype=np.int32)
    n = np.array([2, 3], dtype=np.int32)
    offA = np.array([0, 16], dtype=np.int64)
    offB = np.array([0, 8], dtype=np.int64)
    buf = np.zeros(256)
    p = buf.ctypes.data
    f = H.hsma_trsm_llnn_vbatched_host
    assert f(0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 0, check=False) == 0                      # empty batch
    assert f(2, 0, 2, m, n, 1.0, p, offA, p, offB, p, check=False) == 2                # dtype unsupported
    assert f(9, 0, 2, m, n, 1.0, p, offA, p, offB, p, check=False) == 1                # dtype unknown
    assert f(0, 5, 2, m, n, 1.0, p, offA, p, offB, p, check=False) == 1                # diag unknown
    assert f(0, 0, 2, m, n, 1.0, 0, offA, p, offB, p, check=False) == 1                # NULL hA
    big = np.array([4, 65], dtype=np.int32)
    assert f(0, 0, 2, big, n, 1.0, p, offA, p, offB, p, check=False) == 2              # m > 64
    neg = np.array([4, -1], dtype=np.int32)
    assert f(0, 0, 2, neg, n, 1.0, p, offA, p, offB, p, check=False) == 1              # m < 0
    overlap = np.array([0, 15], dtype=np.int64)                                        # A_0 holds 16 elements
    assert f(0, 0, 2, m, n, 1.0, p, overlap, p, offB, p, check=False) == 1
    assert f(0, 0, 2, m, n, 1.0, p, offA, p, offB, p, chunks=-1, check=False) == 1


def test_fp32_dtypes_plan_and_cost(H):
    """HSMA_R32 and HSMA_C64 use the small direct solve up to m = 64, the blocked path above."""
    for code in (H.R32, H.C64):
        assert H.hsma_plan(code, 64, 100).path == H.PATH_SMALL
        assert H.hsma_plan(code, 65, 1).path == H.PATH_BLOCKED
        assert H.hsma_small_cost(code, 40, 40, 2) > 0
    # the complex dtypes share the complex cost (four FMAs per multiply-add)
    assert H.hsma_small_cost(H.C64, 40, 40, 2) == H.hsma_small_cost(H.C128, 40, 40, 2)
    assert H.hsma_small_cost(H.R32, 40, 40, 2) == H.hsma_small_cost(H.R64, 40, 40, 2)
    assert H.hsma_trsm_llnn(6, 0, 4, 4, 1.0, 1, 4, 1, 4, check=False) == 1  # unknown dtype


def test_variant_argument_checks(H):
    """hsma_trsm validates side / uplo / trans / diag and the leading dimension of A by side."""
    f = H.hsma_trsm
    assert f(0, 2, 0, 0, 0, 4, 4, 1.0, 1, 4, 1, 4, check=False) == 1   # side
    assert f(0, 0, 2, 0, 0, 4, 4, 1.0, 1, 4, 1, 4, check=False) == 1   # uplo
    assert f(0, 0, 0, 3, 0, 4, 4, 1.0, 1, 4, 1, 4, check=False) == 1   # trans
    assert f(0, 0, 0, 1, 2, 4, 4, 1.0, 1, 4, 1, 4, check=False) == 1   # diag
    assert f(9, 0, 0, 1, 0, 4, 4, 1.0, 1, 4, 1, 4, check=False) == 1   # dtype
    assert f(0, 1, 0, 0, 0, 4, 9, 1.0, 1, 8, 1, 4, check=False) == 1   # right side: lda < n
    assert f(0, 0, 1, 0, 0, 4, 9, 1.0, 1, 3, 1, 4, check=False) == 1   # left side: lda < m
    assert f(0, 1, 1, 2, 0, 0, 9, 1.0, 0, 9, 0, 1, check=False) == 0   # m = 0: quick return
    assert f(0, 1, 1, 2, 0, 4, 4, 1.0, 0, 4, 1, 4, check=False) == 1   # NULL A


def test_batched_variant_argument_checks(H):
    f = H.hsma_trsm_vbatched
    assert f(0, 1, 0, 0, 0, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 2   # right side: not batched
    assert f(0, 0, 3, 0, 0, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 1   # uplo
    assert f(0, 0, 1, 5, 0, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 1   # trans
    assert f(2, 0, 1, 1, 0, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 2   # dtype without a small path
    assert f(0, 0, 1, 1, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, check=False) == 0   # empty batch


def test_wait_check_argument_checks(H):
    f = H.hsma_check_wait_timeout
    assert f(10_000_000, 0, check=False) == 1          # NULL result pointer
    assert f(999_999, 0x1000, check=False) == 1        # limit below 1 ms
    assert f(2_000_000_001, 0x1000, check=False) == 1  # limit above 2 s


def test_getrs_argument_checks(H):
    f = H.hsma_getrs_vbatched
    assert f(2, 4, 1, 1, 1.0, 1, 1, 0, 1, 1, check=False) == 2              # dtype without a small path
    assert f(9, 4, 1, 1, 1.0, 1, 1, 0, 1, 1, check=False) == 1              # unknown dtype
    assert f(0, 4, 1, 1, 1.0, 0, 1, 0, 1, 1, max_m=65, check=False) == 1    # NULL LU, large instances allowed
    assert f(0, -1, 1, 1, 1.0, 1, 1, 0, 1, 1, check=False) == 1             # negative batch
    assert f(0, 4, 1, 1, 1.0, 0, 1, 0, 1, 1, check=False) == 1              # NULL LU
    assert f(0, 0, 0, 0, 1.0, 0, 0, 0, 0, 0, check=False) == 0              # empty batch


def test_potrs_argument_checks(H):
    f = H.hsma_potrs_vbatched
    assert f(3, 4, 1, 1, 1.0, 1, 1, 1, 1, check=False) == 2              # dtype without a small path
    assert f(0, 4, 1, 1, 1.0, 1, 1, 0, 1, max_m=65, check=False) == 1    # NULL B, large instances allowed
    assert f(1, 4, 1, 1, 1.0, 1, 1, 0, 1, check=False) == 1              # NULL B
    assert f(1, 0, 0, 0, 1.0, 0, 0, 0, 0, check=False) == 0              # empty batch


def test_single_factor_solve_argument_checks(H):
    assert H.hsma_getrs(9, 4, 4, 1.0, 1, 4, 0, 1, 4, check=False) == 1     # unknown dtype
    assert H.hsma_getrs(0, 4, 4, 1.0, 1, 3, 0, 1, 4, check=False) == 1     # lda < m
    assert H.hsma_getrs(0, 4, 4, 1.0, 0, 4, 0, 1, 4, check=False) == 1     # NULL LU
    assert H.hsma_getrs(0, 0, 4, 1.0, 0, 1, 0, 0, 1, check=False) == 0     # m = 0: no-op
    assert H.hsma_potrs(1, 4, -1, 1.0, 1, 4, 1, 4, check=False) == 1       # n < 0
    assert H.hsma_potrs(1, 4, 4, 1.0, 1, 4, 1, 2, check=False) == 1        # ldb < m
    assert H.hsma_potrs(1, 5, 0, 1.0, 0, 5, 0, 5, check=False) == 0        # n = 0: no-op


def test_header_is_plain_c(tmp_path):
    """include/hsma.h is a C ABI: it compiles as strict C99 (and as C++), with no torch or
    CUDA types in any signature."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = os.path.join(root, "include", "hsma.h")
    code = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)  # declarations only
    assert "torch" not in code and "cudaStream_t" not in code and "at::" not in code
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    src = tmp_path / "c.c"
    src.write_text('#include "hsma.h"\nint main(void) { return (int)(sizeof(hsma_opts_t) == 0); }\n')
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([gcc, "-x", lang, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                            "-I", os.path.dirname(hdr), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_tuning_table_full_configuration(H, tmp_path):
    """Section 4.3.2's table carries the whole blocked configuration: N_B, the FP64
    product tile, split K and the update direction per (dtype, m, n), and N_B and the
    update-panel width of the emulated-products path (table keys dtype + 10); the planner
    reports the nearest entry's fields, options override them."""
    f = tmp_path / "t.txt"
    f.write_text("# dtype m n nb tile split_k looking panel_cols\n"
                 "0 1000 1000 128 2 2 2 2048\n"
                 "0 8000 8000 512 1 1 1 2048\n"
                 "10 8000 8000 256 0 1 1 3072\n"
                 "1 1000 100 64 3 1 2 2048\n")
    try:
        assert H.hsma_tuning_load(str(f)) == 0
        p = H.hsma_plan(H.R64, 900, 1100)
        assert (p.nb, p.tile, p.split_k, p.looking) == (128, H.TILE_128x16, H.SPLITK_OFF, H.LOOK_LEFT)
        p = H.hsma_plan(H.R64, 9000, 9000)
        assert (p.nb, p.tile, p.split_k, p.looking) == (512, H.TILE_64x64, H.SPLITK_AUTO, H.LOOK_RIGHT)
        p = H.hsma_plan(H.C128, 1000, 100)
        assert (p.nb, p.tile, p.looking) == (64, H.TILE_128x8, H.LOOK_LEFT)
        # the emulated entries are not used by the plain FP64 plan
        assert H.hsma_plan(H.R64, 8000, 8000).nb == 512
        for bad in ("0 100 100 64 4 1 1 2048\n", "0 100 100 64 1 3 1 2048\n", "0 100 100 64 1 1 0 2048\n",
                    "0 100 100 64 1 1 1 100\n", "0 100 100 64 1 1\n", "12 100 100 64\n"):
            b = tmp_path / "bad.txt"
            b.write_text(bad)
            assert H.hsma_tuning_load(str(b)) == 1, bad
        assert H.hsma_plan(H.R64, 900, 1100).nb == 128  # unchanged after rejected loads
    finally:
        assert H.hsma_tuning_load(None) == 0


@pytest.mark.parametrize("field,value", [("tile", 4), ("tile", -1), ("split_k", 3), ("looking", 3),
                                         ("panel_cols", 100), ("panel_cols", 8256), ("nb", 40)])
def test_blocked_options_validated(H, field, value):
    """Out-of-range blocked-path options are argument errors, found before any launch."""
    o = H.Opts()
    setattr(o, field, value)
    s = H.hsma_trsm_llnn_ex(H.R64, 0, 200, 10, 1.0, 16, 200, 16, 200, 0, opts=o, check=False)
    assert s == 1
