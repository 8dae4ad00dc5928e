"""Small-case path (m <= 64) and varlen batch against the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2608_25469_gb300 import inputs as I
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative Frobenius forward error, fp64 and complex128
R32, C64 = 4, 5  # the C ABI's FP32 dtype codes (the generators draw FP64 values, rounded)


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available()
    return U.lib()


def _np_dt(code):
    return np.float64 if code == I.R64 else np.complex128


def _solve_single(H, code, A, B, alpha, unit=False, groups=0):
    """A: (lda, m) Fortran, B: (ldb, n) Fortran; returns the device result as numpy."""
    import torch
    dA, dB = H.to_device(A), H.to_device(B)
    opts = H.Opts()
    opts.groups = groups
    H.hsma_trsm_llnn_ex(code, int(unit), A.shape[1], B.shape[1], alpha, dA.data_ptr(), A.shape[0], dB.data_ptr(),
                        B.shape[0], H.stream_ptr(), opts=opts)
    torch.cuda.synchronize()
    return H.from_device(dB)


def test_config0_single_fp64_64(H):
    """One fp64 solve, m = n = 64, lda = ldb = 64, alpha = 1.5, seed 0."""
    A, B = I.gen_A(0, 64, I.R64), I.gen_B(0, 64, 64, I.R64)
    X = _solve_single(H, I.R64, A, B, 1.5)
    ref = oracle.solve(A, B, 1.5)
    assert oracle.forward_error(X, ref) <= TOL
    assert oracle.backward_error(A, B, X, 1.5) <= 1e-14


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_small_sweep_every_m_and_variant(H, code):
    """Every m in 1..64, ragged n, every row-group variant the single path has."""
    import torch
    rng = np.random.default_rng(11)
    dt = _np_dt(code)
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    cases = []
    for m in range(1, 65):
        for n in (1, 5, 33, 64, 97):
            for g in (0, 1, 2, 4, 8, 16, 32):
                if g and H.hsma_small_cost(code, m, n, g) < 0:
                    continue
                cases.append((m, n, g))
    # fixed inputs per (m, n); all launches on one stream, one sync
    data = {}
    jobs = []
    for (m, n, g) in cases:
        if (m, n) not in data:
            seed = int(rng.integers(1 << 30))
            data[(m, n)] = (I.gen_A(seed, m, code), I.gen_B(seed, m, n, code))
        A, B = data[(m, n)]
        dA, dB = H.to_device(A), H.to_device(B)
        opts = H.Opts()
        opts.groups = g
        H.hsma_trsm_llnn_ex(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr(), opts=opts)
        jobs.append((m, n, g, dA, dB))
    torch.cuda.synchronize()
    refs = {k: oracle.solve(A, B, alpha) for k, (A, B) in data.items()}
    worst = 0.0
    for (m, n, g, dA, dB) in jobs:
        err = oracle.forward_error(H.from_device(dB), refs[(m, n)])
        worst = max(worst, err)
        assert err <= TOL, (m, n, g, err)
    assert worst < 1e-14


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_poison_and_canaries(H, code):
    """Upper triangle and (unit) diagonal are never read; padding rows of B are never written."""
    dt = _np_dt(code)
    m, n, pad = 45, 19, 5
    alpha = 0.5 if code == I.R64 else 0.5 + 2j
    A0, B0 = I.gen_A(3, m, code), I.gen_B(3, m, n, code)
    A = np.full((m + pad, m), np.nan, dtype=dt, order="F")
    A[:m] = A0
    A[:m][np.triu_indices(m, 1)] = np.nan
    Bb = I.embed(B0, m + pad, fill=np.nan)
    X = _solve_single(H, code, A, Bb, alpha)
    assert np.all(np.isnan(X[m:])), "padding rows of B were written"
    ref = oracle.solve(A0, B0, alpha)
    assert oracle.forward_error(X[:m], ref) <= TOL
    # unit diagonal: diagonal holds NaN and must not be read
    Au = np.array(A, order="F")
    np.fill_diagonal(Au[:m], np.nan)
    Xu = _solve_single(H, code, Au, Bb, alpha, unit=True)
    A1 = np.array(A0, order="F")
    np.fill_diagonal(A1, 1.0)
    refu = oracle.solve(A1, B0, alpha)
    assert oracle.forward_error(Xu[:m], refu) <= TOL
    # alpha = 0: B := 0, A not read
    Anan = np.full((m, m), np.nan, dtype=dt, order="F")
    X0 = _solve_single(H, code, Anan, Bb, 0.0)
    assert np.all(X0[:m] == 0) and np.all(np.isnan(X0[m:]))


@pytest.mark.parametrize("code", [I.R64, I.C128, R32, C64])
@pytest.mark.parametrize("unit", [False, True])
def test_full_size_single_equals_other_variants(H, code, unit):
    """m = 64 with the 32-row-group variant runs the full-size kernel (one-pass
    staging, B loaded before it); every variant does the same multiply-adds per row in
    the same order, so it equals the 8-row-group variant bit for bit.  Padding rows of
    A and its upper triangle (and, for a unit diagonal, the diagonal) hold NaN and are
    never read; padding rows of B are never written; n = 10000 gives some warps a
    second column tile."""
    m, pad = 64, 6
    dt = {I.R64: np.float64, I.C128: np.complex128, R32: np.float32, C64: np.complex64}[code]
    gcode = I.R64 if code in (I.R64, R32) else I.C128
    alpha = 1.5 if gcode == I.R64 else 1.5 - 0.5j
    A0 = I.gen_A(21, m, gcode).astype(dt)
    A = np.full((m + pad, m), np.nan, dtype=dt, order="F")
    A[:m] = A0
    A[:m][np.triu_indices(m, 1)] = np.nan
    if unit:
        np.fill_diagonal(A[:m], np.nan)
    for n in (1, 64, 300, 10000):
        B0 = I.gen_B(21, m, n, gcode).astype(dt)
        Bb = I.embed(B0, m + pad, fill=np.nan)
        X = _solve_single(H, code, A, Bb, alpha, unit=unit, groups=32)
        Y = _solve_single(H, code, A, Bb, alpha, unit=unit, groups=8)
        assert np.all(np.isnan(X[m:])), n
        assert np.array_equal(X[:m], Y[:m]), n
        A1 = np.array(A0, order="F").astype(np.complex128 if gcode == I.C128 else np.float64)
        A1[np.triu_indices(m, 1)] = 0
        if unit:
            np.fill_diagonal(A1, 1.0)
        cols = slice(0, min(n, 300))
        ref = oracle.solve(A1, np.asfortranarray(B0[:, cols].astype(A1.dtype)), alpha)
        tol = TOL if code in (I.R64, I.C128) else 2e-5
        assert oracle.forward_error(X[:m, cols].astype(ref.dtype), ref) <= tol, n


def _config1(code=I.C128, batch=8192, seed=0):
    ms, ns = I.batched_sizes(seed, batch)
    As = [I.gen_A(seed, int(m), code, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(seed, int(m), int(n), code, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    return As, Bs


def _run_batch(H, code, As, Bs, alpha, unit=False, max_m=64):
    import torch
    bt = U.Batch(As, Bs)
    H.hsma_trsm_llnn_vbatched(code, int(unit), bt.batch, bt.args()[0], bt.args()[1], alpha, bt.args()[2],
                              bt.args()[3], bt.args()[4], bt.args()[5], max_m=max_m, max_n=0,
                              d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    return bt


def test_config1_batched_c128_parity(H):
    """8192 complex128 instances, m, n uniform in [8, 64], alpha = (1.5, -0.5), one varlen launch."""
    alpha = 1.5 - 0.5j
    As, Bs = _config1()
    bt = _run_batch(H, I.C128, As, Bs, alpha)
    assert bt.status() == 0
    Xs = bt.results()
    refs = oracle.solve_batch(As, Bs, alpha)
    errs = [oracle.forward_error(X, R) for X, R in zip(Xs, refs)]
    assert max(errs) <= TOL, max(errs)


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_batched_alone_equals_in_mix(H, code):
    """Each instance solved alone is bit-identical to its result inside the batch."""
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    As, Bs = _config1(code, batch=300, seed=5)
    mix = _run_batch(H, code, As, Bs, alpha).results()
    refs = oracle.solve_batch(As, Bs, alpha)
    for b in range(0, 300, 7):
        alone = _run_batch(H, code, [As[b]], [Bs[b]], alpha).results()[0]
        assert np.array_equal(alone, mix[b]), b
        assert oracle.forward_error(mix[b], refs[b]) <= TOL


def test_batched_edge_instances(H):
    """Empty instances are skipped; invalid ones are skipped and flagged; the rest are solved."""
    code = I.R64
    alpha = -2.0
    As, Bs = [], []
    for m, n in [(5, 3), (0, 4), (7, 0), (64, 64), (1, 1), (13, 29)]:
        As.append(I.gen_A(9, m, code) if m else np.zeros((0, 0), order="F"))
        Bs.append(I.gen_B(9, m, n, code) if m else np.zeros((0, n), order="F"))
    bt = _run_batch(H, code, As, Bs, alpha)
    assert bt.status() == 0
    for A, B, X in zip(As, Bs, bt.results()):
        if A.shape[1] == 0 or B.shape[1] == 0:
            continue
        assert oracle.forward_error(X, oracle.solve(A, B, alpha)) <= TOL
    # an instance with m > 64 and one with ldb < m: skipped, flagged
    import torch
    As2 = [I.gen_A(1, 8, code), I.gen_A(1, 8, code)]
    Bs2 = [I.gen_B(1, 8, 3, code), I.gen_B(1, 8, 3, code)]
    bt = U.Batch(As2, Bs2)
    bt.d_m[1] = 80
    H.hsma_trsm_llnn_vbatched(code, 0, 2, *bt.args()[:2], alpha, *bt.args()[2:], max_m=0, max_n=0,
                              d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    assert bt.status() & H.DEVERR_BAD_SIZE
    X = bt.results()
    assert oracle.forward_error(X[0], oracle.solve(As2[0], Bs2[0], alpha)) <= TOL
    assert np.array_equal(X[1], Bs2[1])  # untouched


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_device_generator_matches_host(H, code):
    import torch
    dt = U.torch_dtype(_np_dt(code))
    for kind, (m, cols), inst in [(0, (37, 37), -1), (1, (37, 11), 4), (0, (64, 64), 12), (2, (45, 45), 3)]:
        ld = m + 3
        t = torch.full((cols, ld), 7.0, dtype=dt, device="cuda")
        H.hsma_gen_matrix(code, kind, 42, inst, m, cols, t.data_ptr(), ld, H.stream_ptr())
        torch.cuda.synchronize()
        got = H.from_device(t)
        ref = {0: lambda: I.gen_A(42, m, code, inst=inst), 1: lambda: I.gen_B(42, m, cols, code, inst=inst),
               2: lambda: I.gen_LU(42, m, code, inst=inst)}[kind]()
        assert np.array_equal(got[:m], ref)
        assert np.all(got[m:] == 7.0)


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("chunks,pinned", [(0, True), (1, True), (3, False), (7, True), (1000, True)])
def test_batched_host_buffers_equal_device_batch(H, code, chunks, pinned):
    """The host-buffer entry point (chunked copies overlapped with the solves) gives the
    device-resident batch's results bit for bit, pinned or pageable host memory."""
    import torch
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    As, Bs = _config1(code, batch=1000, seed=11)
    dev = _run_batch(H, code, As, Bs, alpha).results()
    ms = np.array([a.shape[1] for a in As], dtype=np.int32)
    ns = np.array([b.shape[1] for b in Bs], dtype=np.int32)
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)[:-1]]).astype(np.int64)
    offB = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]]).astype(np.int64)
    hA = np.concatenate([a.ravel(order="F") for a in As])
    hB = np.concatenate([b.ravel(order="F") for b in Bs])
    if pinned:
        tA, tB = torch.from_numpy(hA).pin_memory(), torch.from_numpy(hB).pin_memory()
        tX = torch.empty_like(tB).pin_memory()
        pA, pB, pX, X = tA.data_ptr(), tB.data_ptr(), tX.data_ptr(), tX
    else:
        hX = np.empty_like(hB)
        pA, pB, pX, X = hA.ctypes.data, hB.ctypes.data, hX.ctypes.data, hX
    H.hsma_trsm_llnn_vbatched_host(code, 0, len(As), ms, ns, alpha, pA, offA, pB, offB, pX, chunks=chunks,
                                   stream=H.stream_ptr())
    torch.cuda.synchronize()
    out = X.numpy() if pinned else X
    for b in range(len(As)):
        got = out[offB[b]:offB[b] + ms[b] * ns[b]].reshape((ms[b], ns[b]), order="F")
        assert np.array_equal(got, dev[b]), b


def test_host_buffers_with_gaps_and_empty_instances(H):
    """Offsets with gaps between instances and instances with m = 0 or n = 0 (skipped):
    the solved instances equal the device batch's results.  Each group of consecutive
    instances is copied as one range, so a gap inside a group receives hB's gap
    elements and a gap between groups (or before the first / after the last
    instance) keeps hX's old contents."""
    import torch
    alpha = 0.5 - 1.5j
    As, Bs = _config1(I.C128, batch=300, seed=12)
    for b in range(0, 300, 37):  # empty instances
        As[b] = np.zeros((0, 0), np.complex128) if b % 2 else As[b]
        Bs[b] = np.zeros((As[b].shape[0], 0), np.complex128) if b % 2 == 0 else np.zeros((0, 0), np.complex128)
    dev = _run_batch(H, I.C128, As, Bs, alpha).results()
    ms = np.array([a.shape[1] for a in As], dtype=np.int32)
    ns = np.array([b.shape[1] for b in Bs], dtype=np.int32)
    gap = 5
    offA = np.concatenate([[3], 3 + np.cumsum(ms.astype(np.int64) ** 2 + gap)[:-1]]).astype(np.int64)
    offB = np.concatenate([[2], 2 + np.cumsum(ms.astype(np.int64) * ns + gap)[:-1]]).astype(np.int64)
    hA = np.full(int(offA[-1] + ms[-1] ** 2 + gap), np.nan, np.complex128)
    hB = np.full(int(offB[-1] + ms[-1] * ns[-1] + gap), np.nan, np.complex128)
    for b in range(len(As)):
        hA[offA[b]:offA[b] + ms[b] ** 2] = As[b].ravel(order="F")
        hB[offB[b]:offB[b] + ms[b] * ns[b]] = Bs[b].ravel(order="F")
    hX = np.full_like(hB, 7.0)
    H.hsma_trsm_llnn_vbatched_host(I.C128, 0, len(As), ms, ns, alpha, hA.ctypes.data, offA, hB.ctypes.data, offB,
                                   hX.ctypes.data, chunks=5, stream=H.stream_ptr())
    torch.cuda.synchronize()
    for b in range(len(As)):
        sl = slice(offB[b], offB[b] + ms[b] * ns[b])
        assert np.array_equal(hX[sl].reshape((ms[b], ns[b]), order="F"), dev[b]), b
    assert np.all(hX[:2] == 7.0) and np.all(hX[-gap:] == 7.0)
    per = -(-len(As) // 5)  # instances per group for chunks = 5
    for b in range(len(As) - 1):
        g = hX[offB[b] + ms[b] * ns[b]:offB[b + 1]]
        assert g.size == gap
        if b // per == (b + 1) // per:  # inside one group: hB's gap elements (NaN)
            assert np.all(np.isnan(g)), b
        else:  # between groups: untouched
            assert np.all(g == 7.0), b


def test_golden_integer_solves_bitwise(H):
    """The integer-valued golden solves (small kernel for m <= 64, blocked path above):
    every intermediate is an integer below 2^53, so the GPU result equals X bit for bit."""
    import torch
    from tests import golden_cases
    for dtype, A, B, alpha, X in golden_cases.load():
        code = I.C128 if dtype == "c128" else I.R64
        m, n = B.shape
        dA, dB = H.to_device(A), H.to_device(B)
        H.hsma_trsm_llnn(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(H.from_device(dB), X), (dtype, m, n)


def _noalloc(H, code, As, Bs, alpha, unit=False):
    """The per-instance batched kernel (the allocation-free entry point runs it)."""
    import torch
    bt = U.Batch(As, Bs)
    H.hsma_trsm_llnn_vbatched_noalloc(code, int(unit), bt.batch, *bt.args()[:2], alpha, *bt.args()[2:], max_m=64,
                                      max_n=0, d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    return bt


def _mix(code, sizes, seed, pad=0):
    dt = {I.R64: np.float64, I.C128: np.complex128, C64: np.complex64, R32: np.float32}[code]
    gcode = I.C128 if code in (I.C128, C64) else I.R64
    As, Bs = [], []
    for b, (m, n) in enumerate(sizes):
        A = I.gen_A(seed, m, gcode, inst=b).astype(dt)
        B = I.gen_B(seed, m, n, gcode, inst=b).astype(dt)
        As.append(I.embed(A, m + pad) if pad else np.asfortranarray(A))
        Bs.append(I.embed(B, m + pad) if pad else np.asfortranarray(B))
    return As, Bs


PACKED_MIXES = {
    # the workload's size mix
    "uniform8_64": lambda rng: [(int(m), int(n)) for m, n in rng.integers(8, 65, (1500, 2))],
    # one column per instance: a warp tile spans 16 or 32 instances
    "n1": lambda rng: [(int(m), 1) for m in rng.integers(1, 65, 900)],
    # wide instances (n > 64) and every m, including 1, 32, 33 and 64
    "wide_every_m": lambda rng: [(m, int(rng.integers(60, 200))) for m in range(1, 65)],
    # a single instance, and groups with one instance each
    "single": lambda rng: [(33, 7)],
    "one_per_m": lambda rng: [(m, (m * 7) % 40 + 1) for m in range(64, 0, -1)],
}


@pytest.mark.parametrize("code", [I.R64, I.C128, C64, R32])
@pytest.mark.parametrize("mix", sorted(PACKED_MIXES))
def test_packed_batch_equals_per_instance_kernel(H, code, mix):
    """The column-packed batch (warps serve columns of several instances of the same m)
    gives the per-instance kernel's results bit for bit, on size mixes that put many
    instances in one warp tile, wide instances, every m and lone instances; and the
    oracle's within the dtype's tolerance."""
    rng = np.random.default_rng(sum(map(ord, mix)))
    sizes = PACKED_MIXES[mix](rng)
    alpha = {I.R64: 1.5, R32: 1.5}.get(code, 1.5 - 0.5j)
    As, Bs = _mix(code, sizes, seed=31)
    got = _run_batch(H, code, As, Bs, alpha)
    ref = _noalloc(H, code, As, Bs, alpha)
    assert got.status() == 0 and ref.status() == 0
    G, R = got.results(), ref.results()
    for b in range(len(As)):
        assert np.array_equal(G[b], R[b]), (mix, b, sizes[b])
    tol = TOL if code in (I.R64, I.C128) else 2e-5
    wide = lambda L: [np.asfortranarray(x.astype(np.complex128 if np.iscomplexobj(x) else np.float64)) for x in L]
    pick = list(range(0, len(As), max(1, len(As) // 60)))
    refs = oracle.solve_batch(wide([As[b] for b in pick]), wide([Bs[b] for b in pick]), alpha)
    for k, b in enumerate(pick):
        assert oracle.forward_error(G[b].astype(refs[k].dtype), refs[k]) <= tol, (mix, b)


def _trsm_vbatched(H, code, uplo, trans, unit, As, Bs, alpha):
    import torch
    bt = U.Batch(As, Bs)
    a = bt.args()
    H.hsma_trsm_vbatched(code, H.LEFT, uplo, trans, int(unit), bt.batch, a[0], a[1], alpha, a[2], a[3], a[4], a[5],
                         64, 0, bt.d_status.data_ptr(), H.stream_ptr())
    torch.cuda.synchronize()
    assert bt.status() == 0
    return bt.results()


@pytest.mark.parametrize("code", [I.R64, I.C128])
@pytest.mark.parametrize("uplo,trans", [(1, 0), (0, 1), (0, 2), (1, 1), (1, 2)])
@pytest.mark.parametrize("unit", [False, True])
def test_mapped_batch_equals_explicit_lower_system(H, code, uplo, trans, unit):
    """Every left-side variant of the varlen batch reads A and B through an index map: op(A)
    (transpose, conjugate transpose), reversed in rows and columns when op(A) is upper.  Its
    results equal the lower / no-transpose batch on that system written out explicitly
    (J op(A) J, J B; X = J X'), bit for bit.  The triangle the variant does not reference
    holds NaN, so it is never read."""
    rng = np.random.default_rng(60 + 10 * uplo + 3 * trans + unit)
    sizes = [(int(m), int(n)) for m, n in rng.integers(1, 65, (700, 2))] + [(m, 3) for m in range(1, 65)]
    alpha = 1.25 if code == I.R64 else 1.25 - 0.75j
    As, Bs = _mix(code, sizes, seed=61 + uplo + trans)
    op_lower = (uplo == 0) != (trans != 0)
    Am, Ae, Be = [], [], []
    for A, B in zip(As, Bs):
        T = A if uplo == 0 else np.asfortranarray(A.T)  # the referenced triangle in place
        T = np.array(T, order="F")
        T[np.triu_indices(T.shape[0], 1) if uplo == 0 else np.tril_indices(T.shape[0], -1)] = np.nan
        Am.append(T)
        op = T if trans == 0 else (T.T if trans == 1 else T.conj().T)
        Ae.append(np.asfortranarray(op if op_lower else op[::-1, ::-1]))
        Be.append(np.asfortranarray(B if op_lower else B[::-1]))
    got = _trsm_vbatched(H, code, uplo, trans, unit, Am, Bs, alpha)
    ref = _noalloc(H, code, Ae, Be, alpha, unit=unit)
    assert ref.status() == 0
    R = ref.results()
    for b in range(len(As)):
        X = R[b] if op_lower else R[b][::-1]
        assert np.array_equal(got[b], X), (b, sizes[b])
        assert not np.isnan(got[b]).any(), b
    for b in range(0, len(As), 97):
        refo = oracle.solve_general(np.nan_to_num(Am[b]), Bs[b], alpha, 0, uplo, trans, unit)
        assert oracle.forward_error(got[b], refo) <= TOL, b


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_packed_batch_padding_unit_and_zero_alpha(H, code):
    """lda, ldb > m: padding rows of B stay untouched and padding rows of A are never
    read (NaN); unit diagonal (NaN on the diagonal, never read); alpha = 0 gives zeros
    without reading A.  Bit-equal to the per-instance kernel."""
    rng = np.random.default_rng(4)
    sizes = [(int(m), int(n)) for m, n in rng.integers(1, 65, (400, 2))]
    As, Bs = _mix(code, sizes, seed=8, pad=3)
    for A in As:
        A[np.triu_indices(A.shape[1], 1)] = np.nan
    alpha = 0.75 if code == I.R64 else 0.25 + 1j
    got = _run_batch(H, code, As, Bs, alpha)
    ref = _noalloc(H, code, As, Bs, alpha)
    for b, (X, Y) in enumerate(zip(got.results(), ref.results())):
        m = sizes[b][0]
        assert np.all(np.isnan(X[m:])), b
        assert np.array_equal(X[:m], Y[:m]), b
    Au = [np.array(A, order="F") for A in As]
    for A in Au:
        np.fill_diagonal(A, np.nan)
    got = _run_batch(H, code, Au, Bs, alpha, unit=True)
    ref = _noalloc(H, code, Au, Bs, alpha, unit=True)
    for b, (X, Y) in enumerate(zip(got.results(), ref.results())):
        m = sizes[b][0]
        assert np.array_equal(X[:m], Y[:m]) and not np.isnan(X[:m]).any(), b
        if b % 50 == 0:
            A1 = np.array(As[b][:m], order="F")
            np.fill_diagonal(A1, 1.0)
            A1[np.triu_indices(m, 1)] = 0
            assert oracle.forward_error(X[:m], oracle.solve(A1, np.asfortranarray(Bs[b][:m]), alpha)) <= TOL
    Anan = [np.full_like(A, np.nan) for A in As]
    got = _run_batch(H, code, Anan, Bs, 0.0)
    for b, X in enumerate(got.results()):
        m = sizes[b][0]
        assert np.all(X[:m] == 0) and np.all(np.isnan(X[m:])), b


def test_packed_batch_instance_above_max_m_is_skipped(H):
    """max_m sizes the staging workspace: an instance with m above it is skipped and
    flagged (HSMA_DEVERR_BAD_SIZE), its B untouched; the others are solved."""
    code = I.C128
    alpha = 2.0 - 1j
    As, Bs = _mix(code, [(20, 9), (40, 5), (17, 33)], seed=3)
    bt = _run_batch(H, code, As, Bs, alpha, max_m=24)
    assert bt.status() & H.DEVERR_BAD_SIZE
    X = bt.results()
    assert np.array_equal(X[1], Bs[1])
    for b in (0, 2):
        assert oracle.forward_error(X[b], oracle.solve(As[b], Bs[b], alpha)) <= TOL


@pytest.mark.parametrize("code", [I.R64, I.C128])
def test_batch_with_instances_above_64(H, code):
    """max_m > 64: instances of any size in one call.  The small ones run as the batch
    (bit-equal to the batch without the large ones), each large one through the
    single-solve path (bit-equal to hsma_trsm_llnn alone); all within the oracle's
    tolerance.  A large instance with ldb < m is skipped and flagged."""
    import torch
    rng = np.random.default_rng(50)
    sizes = [(int(m), int(n)) for m, n in rng.integers(1, 65, (120, 2))]
    for k, mm in zip((3, 40, 77, 100), (65, 130, 300, 700)):
        sizes[k] = (mm, int(rng.integers(1, 90)))
    alpha = 1.5 if code == I.R64 else 1.5 - 0.5j
    As, Bs = _mix(code, sizes, seed=51)
    got = _run_batch(H, code, As, Bs, alpha, max_m=1000)
    assert got.status() == 0
    G = got.results()
    small = [b for b, (m, _) in enumerate(sizes) if m <= 64]
    only = _run_batch(H, code, [As[b] for b in small], [Bs[b] for b in small], alpha).results()
    for k, b in enumerate(small):
        assert np.array_equal(G[b], only[k]), b
    for b, (m, n) in enumerate(sizes):
        if m > 64:
            dA, dB = H.to_device(As[b]), H.to_device(Bs[b])
            H.hsma_trsm_llnn(code, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, H.stream_ptr())
            torch.cuda.synchronize()
            assert np.array_equal(G[b], H.from_device(dB)), b
        assert oracle.forward_error(G[b], oracle.solve(As[b], Bs[b], alpha)) <= TOL, b
    # a large instance whose ldb is too small: skipped, flagged, B untouched
    bt = U.Batch(As[:5], Bs[:5])
    bt.d_ldb[3] = 10
    H.hsma_trsm_llnn_vbatched(code, 0, 5, *bt.args()[:2], alpha, *bt.args()[2:], max_m=200, max_n=0,
                              d_status=bt.d_status.data_ptr(), stream=H.stream_ptr())
    torch.cuda.synchronize()
    assert bt.status() & H.DEVERR_BAD_SIZE
    assert np.array_equal(bt.results()[3], Bs[3])


def test_factor_batches_with_instances_above_64(H):
    """LU- and Cholesky-factor batches with max_m > 64: large instances through hsma_getrs /
    hsma_potrs, against the oracle's getrs / potrs."""
    import torch
    code = I.C128
    rng = np.random.default_rng(52)
    sizes = [(int(m), int(n)) for m, n in rng.integers(4, 65, (40, 2))] + [(90, 7), (257, 33)]
    Fs = [I.gen_LU(53, m, code, inst=b) for b, (m, _) in enumerate(sizes)]
    Bs = [I.gen_B(53, m, n, code, inst=b) for b, (m, n) in enumerate(sizes)]
    pivs = [np.array([int(rng.integers(k, m)) + 1 for k in range(m)], dtype=np.int32) for m, _ in sizes]
    dpiv = [torch.from_numpy(p).cuda() for p in pivs]
    pp = torch.tensor([p.data_ptr() for p in dpiv], dtype=torch.int64, device="cuda")
    bt = U.Batch(Fs, Bs)
    H.hsma_getrs_vbatched(code, bt.batch, bt.d_m.data_ptr(), bt.d_n.data_ptr(), 0.5 + 0.5j, bt.d_ptrA.data_ptr(),
                          bt.d_lda.data_ptr(), pp.data_ptr(), bt.d_ptrB.data_ptr(), bt.d_ldb.data_ptr(), 300, 0,
                          bt.d_status.data_ptr(), H.stream_ptr())
    torch.cuda.synchronize()
    assert bt.status() == 0
    for b, X in enumerate(bt.results()):
        assert oracle.forward_error(X, oracle.getrs(Fs[b], pivs[b], Bs[b], 0.5 + 0.5j)) <= TOL, b
    Ls = [I.gen_A(54, m, code, inst=b) for b, (m, _) in enumerate(sizes)]
    bt = U.Batch(Ls, Bs)
    H.hsma_potrs_vbatched(code, bt.batch, bt.d_m.data_ptr(), bt.d_n.data_ptr(), 2.0, bt.d_ptrA.data_ptr(),
                          bt.d_lda.data_ptr(), bt.d_ptrB.data_ptr(), bt.d_ldb.data_ptr(), 300, 0,
                          bt.d_status.data_ptr(), H.stream_ptr())
    torch.cuda.synchronize()
    assert bt.status() == 0
    for b, X in enumerate(bt.results()):
        assert oracle.forward_error(X, oracle.potrs(Ls[b], Bs[b], 2.0)) <= TOL, b


def _pack_lower(A):
    """LAPACK's packed lower format: column j's rows j..m-1, one column after the other."""
    m = A.shape[1]
    return np.concatenate([A[j:m, j] for j in range(m)]) if m else np.zeros(0, A.dtype)


@pytest.mark.parametrize("code", [I.R64, I.C128, C64, R32])
@pytest.mark.parametrize("chunks", [0, 3])
def test_host_batch_packed_triangles_equal_square_layout(H, code, chunks):
    """The host-buffer batch with A as packed lower triangles gives the square-layout call's
    results bit for bit; gaps between instances and empty instances included."""
    import torch
    rng = np.random.default_rng(60 + code)
    sizes = [(int(m), int(n)) for m, n in rng.integers(0, 65, (300, 2))]
    As, Bs = _mix(code, [(max(m, 1), max(n, 1)) for m, n in sizes], seed=61)
    As = [a[:m, :m] if m else np.zeros((0, 0), a.dtype) for a, (m, _) in zip(As, sizes)]
    Bs = [b[:m, :n] for b, (m, n) in zip(Bs, sizes)]
    alpha = 1.5 if code in (I.R64, R32) else 1.5 - 0.5j
    ms = np.array([m for m, _ in sizes], dtype=np.int32)
    ns = np.array([n for _, n in sizes], dtype=np.int32)
    gap = 3
    sqA = ms.astype(np.int64) ** 2
    tpA = ms.astype(np.int64) * (ms + 1) // 2
    nB = ms.astype(np.int64) * ns
    offS = np.concatenate([[0], np.cumsum(sqA)[:-1]]).astype(np.int64)
    offT = np.concatenate([[5], 5 + np.cumsum(tpA + gap)[:-1]]).astype(np.int64)
    offB = np.concatenate([[0], np.cumsum(nB + gap)[:-1]]).astype(np.int64)
    dt = As[0].dtype
    hS = np.zeros(int(sqA.sum()) + 1, dt)
    hT = np.full(int(offT[-1] + tpA[-1] + gap), np.nan, dt)
    hB = np.zeros(int(offB[-1] + nB[-1] + gap), dt)
    for b in range(len(sizes)):
        m, n = sizes[b]
        hS[offS[b]:offS[b] + m * m] = np.asfortranarray(As[b]).ravel(order="F")
        hT[offT[b]:offT[b] + tpA[b]] = _pack_lower(As[b])
        hB[offB[b]:offB[b] + m * n] = np.asfortranarray(Bs[b]).ravel(order="F")
    X1, X2 = np.zeros_like(hB), np.zeros_like(hB)
    H.hsma_trsm_llnn_vbatched_host(code, 0, len(sizes), ms, ns, alpha, hS.ctypes.data, offS, hB.ctypes.data, offB,
                                   X1.ctypes.data, chunks=chunks, stream=H.stream_ptr())
    H.hsma_trsm_llnn_vbatched_host_tp(code, 0, len(sizes), ms, ns, alpha, hT.ctypes.data, offT, hB.ctypes.data,
                                      offB, X2.ctypes.data, chunks=chunks, stream=H.stream_ptr())
    torch.cuda.synchronize()
    for b in range(len(sizes)):
        m, n = sizes[b]
        sl = slice(offB[b], offB[b] + m * n)
        assert np.array_equal(X1[sl], X2[sl]), b
    # offsets that overlap the previous packed triangle are rejected before any copy
    bad = offT.copy()
    k = int(np.argmax(tpA > 1))
    if k + 1 < len(bad):
        bad[k + 1] = bad[k] + tpA[k] - 1
        assert H.hsma_trsm_llnn_vbatched_host_tp(code, 0, len(sizes), ms, ns, alpha, hT.ctypes.data, bad,
                                                 hB.ctypes.data, offB, X2.ctypes.data, check=False) == 1
