"""Seeded input generator: SplitMix64 test vector and the workload recipe's structure."""
import numpy as np

from paper_2608_25469_gb300 import inputs as I


def test_splitmix64_reference_vector():
    # First outputs of SplitMix64 from state 1234567 (Vigna's reference generator).
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    got = [I._mix64_int(1234567 + (i + 1) * I.G) for i in range(5)]
    assert got == expected


def test_counter_based_matches_sequential():
    k = I.key(5, I.stream_id(I.B_RE, 3))
    idx = np.arange(10, dtype=np.uint64)
    seq = [I._mix64_int(k + (i + 1) * I.G) for i in range(10)]
    assert [int(v) for v in I.u64(5, I.stream_id(I.B_RE, 3), idx)] == seq


def test_uniform_range_and_moments():
    u = I.u01(0, 1, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002


def test_gen_A_structure():
    for dt in (I.R64, I.C128):
        m = 37
        A = I.gen_A(0, m, dt)
        assert A.flags.f_contiguous and A.shape == (m, m)
        assert np.all(np.triu(A, 1) == 0)
        d = np.diag(A)
        for part in ([d.real, d.imag] if dt == I.C128 else [d]):
            assert np.all((part >= 1.0) & (part < 2.0))
        off = A[np.tril_indices(m, -1)]
        for part in ([off.real, off.imag] if dt == I.C128 else [off]):
            assert np.all(np.abs(part) <= 1.0 / m)


def test_streams_are_distinct():
    a = I.gen_B(0, 8, 8, I.R64, inst=0)
    b = I.gen_B(0, 8, 8, I.R64, inst=1)
    c = I.gen_B(1, 8, 8, I.R64, inst=0)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(a, I.gen_B(0, 8, 8, I.R64, inst=0))


def test_batched_sizes_range():
    m, n = I.batched_sizes(0, 8192)
    assert m.min() == 8 and m.max() == 64 and n.min() == 8 and n.max() == 64
    assert abs(m.mean() - 36) < 1.0 and abs(n.mean() - 36) < 1.0


def test_serving_stream():
    t, m, n, dt = I.serving_requests(0, 20000)
    assert m.min() >= 16 and m.max() <= 4096 and n.min() >= 1 and n.max() <= 512
    assert np.all(np.diff(t) >= 0)
    assert abs(20000 / t[-1] - 2000) < 60
    assert abs((dt == I.R64).mean() - 0.7) < 0.02


def test_gen_B_cols_matches_gen_B():
    B = I.gen_B(4, 29, 13, I.C128, inst=2)
    cols = [0, 12, 5]
    assert np.array_equal(I.gen_B_cols(4, 29, cols, I.C128, inst=2), B[:, cols])


def test_gen_lu_packs_two_triangles():
    """Packed LU factors: below the diagonal gen_A's multipliers (same streams), on and
    above it the transpose of a triangle drawn from the U streams (diagonal in [1, 2),
    off-diagonal entries (2u - 1)/m)."""
    for code in (I.R64, I.C128):
        m = 23
        F = I.gen_LU(5, m, code, inst=2)
        A = I.gen_A(5, m, code, inst=2)
        low = np.tril_indices(m, -1)
        assert np.array_equal(F[low], A[low])
        U = np.triu(F)
        d = np.diag(U)
        assert np.all((d.real >= 1) & (d.real < 2))
        up = np.triu_indices(m, 1)
        assert np.all(np.abs(U[up].real) <= 1.0 / m)
        assert not np.array_equal(np.triu(F, 1).T[low], A[low])  # a different draw
