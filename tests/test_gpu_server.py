"""GPU: the continuous-batching server returns, for every request, exactly what the CPU
oracle returns for that code (d and the canonical witness), and what md_compute returns for it
alone, while requests join and leave the running mix."""
import os
import time

import numpy as np
import pytest

import oracle as O
from paper_1911_08963_gb300 import inputs as I
from tests import textbook as T

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def B():
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding
    return binding


def single(B, G, n, k):
    h = B.md_create(G, n, k)
    try:
        return B.md_compute(h, n)
    finally:
        B.md_destroy(h)


def assert_oracle(G, n, k, d, wit):
    ref = O.bz(G, n, k, threads=THREADS)
    assert d == ref.d and np.array_equal(wit, ref.witness), (n, k, d, ref.d)


def wait(B, s, ticket, n, timeout=120):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = B.md_server_poll(s, ticket, n)
        if r is not None:
            return r
        time.sleep(0.0005)
    raise TimeoutError("request %d did not finish" % ticket)


def test_server_results_equal_alone(B):
    s = B.md_server_create(slots=8)
    try:
        codes = [(T.pack(T.random_rows(n, k, 300 + i), n), n, k)
                 for i, (n, k) in enumerate([(100, 40), (48, 16), (64, 18), (126, 42), (31, 10), (90, 45),
                                             (80, 38), (150, 14), (20, 7), (66, 12), (57, 19), (96, 44)])]
        # a large code first, then the others arrive while it runs
        tickets = [B.md_server_submit(s, G, n, k) for G, n, k in codes]
        out = [wait(B, s, t, n) for t, (G, n, k) in zip(tickets, codes)]
        for (G, n, k), (d, wit, st) in zip(codes, out):
            assert st == B.MD_OK
            assert_oracle(G, n, k, d, wit)
            ds, ws = single(B, G, n, k)
            assert d == ds and np.array_equal(wit, ws)
        # a ticket is returned once
        with pytest.raises(B.MDError):
            B.md_server_poll(s, tickets[0], codes[0][1])
    finally:
        B.md_server_destroy(s)


def test_server_overlap_small_finishes_before_large(B):
    """A small code submitted while a large one (~2e12 combinations) runs is admitted into the
    running mix and finishes first; the small result equals the oracle's, and both equal
    md_compute's (the large one is beyond the oracle in test time)."""
    s = B.md_server_create(slots=4)
    try:
        n, k = 176, 88
        G = T.pack(T.random_rows(n, k, 5), n)
        tl = B.md_server_submit(s, G, n, k)
        time.sleep(0.01)
        small = (T.pack(T.random_rows(40, 12, 9), 40), 40, 12)
        ts = B.md_server_submit(s, *small)
        d_small = wait(B, s, ts, 40)
        assert B.md_server_poll(s, tl, n) is None          # the large code is still running
        d_large = wait(B, s, tl, n)
        assert d_small[2] == B.MD_OK and d_large[2] == B.MD_OK
        assert_oracle(*small, d_small[0], d_small[1])
        assert d_small[0] == single(B, *small)[0]
        ds, ws = single(B, G, n, k)
        assert d_large[0] == ds and np.array_equal(d_large[1], ws)
    finally:
        B.md_server_destroy(s)


def test_server_rejections(B):
    s = B.md_server_create(slots=2, work_budget=10 ** 9)
    try:
        G, n, k = I.single_code("rand200x100")
        with pytest.raises(B.MDError) as e:
            B.md_server_submit(s, G, n, k)
        assert e.value.code == B.MD_EBUDGET
        rows = T.random_rows(30, 8, 7)
        with pytest.raises(B.MDError) as e:
            B.md_server_submit(s, T.pack(rows[:7] + [rows[0] ^ rows[1]], 30), 30, 8)
        assert e.value.code == B.MD_ERANK
        with pytest.raises(B.MDError):
            B.md_server_poll(s, 12345, 30)
    finally:
        B.md_server_destroy(s)


def test_server_trace_sample(B):
    """First requests of the Poisson trace with a work budget (requests whose estimated work
    exceeds it are refused at submission): every accepted one equals the oracle and
    md_compute."""
    s = B.md_server_create(slots=16, work_budget=3 * 10 ** 9)
    try:
        trace = I.serving_trace(40)
        tickets = []
        for t, G, n, k in trace:
            try:
                tickets.append((B.md_server_submit(s, G, n, k), G, n, k))
            except B.MDError as e:
                assert e.code == B.MD_EBUDGET
        assert tickets
        outs = [wait(B, s, tk, n) for tk, G, n, k in tickets]
        for (tk, G, n, k), (d, wit, st) in zip(tickets, outs):
            assert st == B.MD_OK
            assert_oracle(G, n, k, d, wit)
            ds, ws = single(B, G, n, k)
            assert d == ds and np.array_equal(wit, ws)
    finally:
        B.md_server_destroy(s)


def test_server_heavy_route_equals_oracle(B):
    """With a low heavy threshold, the heavier requests of the trace run as single-code
    computations on the server's second worker while the others share the slots; every result
    equals the oracle and md_compute."""
    s = B.md_server_create(slots=8, work_budget=3 * 10 ** 9, heavy=10 ** 7)
    try:
        tickets = []
        for t, G, n, k in I.serving_trace(40):
            try:
                tickets.append((B.md_server_submit(s, G, n, k), G, n, k))
            except B.MDError as e:
                assert e.code == B.MD_EBUDGET
        outs = [wait(B, s, tk, n) for tk, G, n, k in tickets]
        for (tk, G, n, k), (d, wit, st) in zip(tickets, outs):
            assert st == B.MD_OK
            assert_oracle(G, n, k, d, wit)
    finally:
        B.md_server_destroy(s)
    # every request in the slots (the threshold out of reach) gives the same answers
    s = B.md_server_create(slots=8, work_budget=3 * 10 ** 9, heavy=2 ** 64 - 1)
    try:
        again = [wait(B, s, B.md_server_submit(s, G, n, k), n) for tk, G, n, k in tickets]
        assert [(d, list(w)) for d, w, st in again] == [(d, list(w)) for d, w, st in outs]
    finally:
        B.md_server_destroy(s)


def test_server_destroy_ends_running_heavy_request(B):
    """md_server_destroy cancels a single-code computation in flight (rand200x100 runs for
    about half a minute) instead of waiting for it to finish."""
    s = B.md_server_create(slots=2)
    G, n, k = I.single_code("rand200x100")
    tk = B.md_server_submit(s, G, n, k)
    time.sleep(1.0)
    assert B.md_server_poll(s, tk, n) is None
    t0 = time.time()
    B.md_server_destroy(s)
    assert time.time() - t0 < 5.0
