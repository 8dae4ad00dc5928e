"""Serving loop's admission and queue logic with the fake-device backend (no GPU)."""
import threading

import numpy as np
import pytest

from tests import gpu_util as U


@pytest.fixture(scope="module")
def H():
    return U.lib()


def _req(H, m, n, dtype=0, seed=0, inst=0):
    r = H.Request()
    r.dtype, r.diag, r.m, r.n = dtype, 0, m, n
    r.alpha[0], r.alpha[1] = 1.0, 0.0
    r.gen_seed, r.gen_inst = seed, inst
    return r


def test_budget_respected_and_requests_overlap(H):
    budget = 64 << 20
    s = H.hsma_server_create(budget, 4, H.SERVER_FAKE_DEVICE)
    rng = np.random.default_rng(0)
    tickets, sizes = [], []
    lock = threading.Lock()

    def submitter(k):
        loc = np.random.default_rng(k)
        for i in range(150):
            m = int(np.exp(loc.uniform(np.log(16), np.log(1025))))
            n = int(np.exp(loc.uniform(0, np.log(257))))
            t = H.hsma_server_submit(s, _req(H, m, n, int(loc.random() < 0.3), 1, i))
            with lock:
                tickets.append(t)
                sizes.append((m, n))

    th = [threading.Thread(target=submitter, args=(k,)) for k in range(2)]
    [t.start() for t in th]
    [t.join() for t in th]
    assert H.hsma_server_drain(s, 60.0) == 0
    st = H.hsma_server_stats(s)
    assert st.submitted == st.completed == 300 == st.admitted
    assert 0 < st.peak_bytes_in_use <= budget
    assert st.bytes_in_use == 0
    # continuous batching: more than one request resident at once
    biggest = max(16 * m * m + 16 * m * n for m, n in sizes)
    assert st.peak_bytes_in_use > biggest
    lats = []
    for t in tickets:
        done, lat, status = H.hsma_server_poll(s, t)
        assert done and status == 0
        lats.append(lat)
    assert min(lats) > 0
    assert H.hsma_server_destroy(s) == 0


def test_request_larger_than_budget_is_rejected(H):
    s = H.hsma_server_create(1 << 20, 2, H.SERVER_FAKE_DEVICE)
    t_small = H.hsma_server_submit(s, _req(H, 32, 8))
    t_big = H.hsma_server_submit(s, _req(H, 4096, 512))
    assert H.hsma_server_drain(s, 30.0) == 0
    assert H.hsma_server_poll(s, t_small)[2] == 0
    done, _, status = H.hsma_server_poll(s, t_big)
    assert done and status == 3  # HSMA_ERR_NO_MEMORY
    assert H.hsma_server_destroy(s) == 0


def test_tight_budget_serialises_without_overcommit(H):
    # budget fits one 512 x 512 request at a time: all still complete, never two at once
    need = 8 * 512 * 512 + 8 * 512 * 64 + 8 * (2 * 256 * 256 + 256 * 64)
    s = H.hsma_server_create(need + 1000, 3, H.SERVER_FAKE_DEVICE)
    ts = [H.hsma_server_submit(s, _req(H, 512, 64, 0, 3, i)) for i in range(20)]
    assert H.hsma_server_drain(s, 30.0) == 0
    st = H.hsma_server_stats(s)
    assert st.completed == 20 and st.peak_bytes_in_use <= need + 1000
    assert H.hsma_server_destroy(s) == 0


def test_invalid_requests(H):
    s = H.hsma_server_create(1 << 20, 1, H.SERVER_FAKE_DEVICE)
    bad = _req(H, 0, 4)
    with pytest.raises(H.HsmaError):
        H.hsma_server_submit(s, bad)
    bad = _req(H, 8, 4, dtype=2)
    with pytest.raises(H.HsmaError):
        H.hsma_server_submit(s, bad)
    assert H.hsma_server_destroy(s) == 0


def test_unknown_server_flags_rejected(H):
    with pytest.raises(H.HsmaError):
        H.hsma_server_create(1 << 20, 1, 0x80)


def test_emulated_flag_accounts_for_its_workspace(H):
    """With FP64 products emulated, a blocked request also reserves the slice buffers:
    a budget that fits the plain request's need is too small for the emulated one."""
    need_plain = 8 * 512 * 512 + 8 * 512 * 64 + 8 * (2 * 256 * 256 + 256 * 64)
    flags = H.SERVER_FAKE_DEVICE | H.SERVER_FP64_EMULATED
    s = H.hsma_server_create(need_plain + 1000, 1, flags)
    t = H.hsma_server_submit(s, _req(H, 512, 64))
    assert H.hsma_server_drain(s, 30.0) == 0
    done, _, status = H.hsma_server_poll(s, t)
    assert done and status == 3  # HSMA_ERR_NO_MEMORY: never fits
    assert H.hsma_server_destroy(s) == 0
    s = H.hsma_server_create(1 << 30, 2, flags)
    ts = [H.hsma_server_submit(s, _req(H, 512, 64, 0, 3, i)) for i in range(4)]
    assert H.hsma_server_drain(s, 30.0) == 0
    assert all(H.hsma_server_poll(s, t)[2] == 0 for t in ts)
    assert H.hsma_server_destroy(s) == 0
