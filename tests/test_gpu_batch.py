"""GPU: many codes in one schedule (md_batch) give the same d and witness as md_compute on
each code alone (itself pinned to the oracle), and as the CPU oracle on the small ones."""
import numpy as np
import pytest

import oracle as O
from paper_1911_08963_gb300 import inputs as I
from tests import textbook as T

pytestmark = pytest.mark.gpu


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


def mixed_codes():
    codes = []
    for i, (n, k) in enumerate([(20, 7), (48, 16), (64, 18), (100, 33), (90, 45), (126, 42), (31, 10), (80, 38),
                                (24, 12), (150, 14), (66, 12), (200, 195), (256, 3), (12, 1), (70, 35)]):
        codes.append((T.pack(T.random_rows(n, k, 100 + i), n), n, k))
    for name in ("hamming7", "golay24", "rm1_5", "parity10", "trivial6"):
        rows, n, k = T.TEXTBOOK[name][0]()
        codes.append((T.pack(rows, n), n, k))
    return codes


@pytest.mark.parametrize("graph", [1, 0])
def test_batch_matches_single_and_oracle(B, graph):
    codes = mixed_codes()
    d, wits, st = B.md_batch(codes, B.md_options_init(use_graph=graph))
    assert st == [B.MD_OK] * len(codes)
    for (G, n, k), di, wi in zip(codes, d, wits):
        ds, ws = single(B, G, n, k)
        assert di == ds and np.array_equal(wi, ws), (n, k)
        res = O.bz(G, n, k, threads=8)
        assert di == res.d and np.array_equal(wi, res.witness), (n, k)


def test_batch_short_plan_horizon_falls_back(B):
    """With plans one stage past the estimate, codes that run longer are finished by
    single-code runs; every result is still md_compute's."""
    codes = mixed_codes()
    d, wits, st = B.md_batch(codes, B.md_options_init(plan_horizon=1))
    assert st == [B.MD_OK] * len(codes)
    for (G, n, k), di, wi in zip(codes, d, wits):
        ds, ws = single(B, G, n, k)
        assert di == ds and np.array_equal(wi, ws), (n, k)


def test_batch_per_code_loop_mode(B):
    codes = mixed_codes()[:8]
    a = B.md_batch(codes)
    b = B.md_batch(codes, B.md_options_init(batch_mode=1))
    assert a[0] == b[0] and a[2] == b[2]
    assert all(np.array_equal(x, y) for x, y in zip(a[1], b[1]))


def test_batch_statuses(B):
    good = mixed_codes()[:3]
    rows = T.random_rows(30, 8, 7)
    bad_rank = (T.pack(rows[:7] + [rows[0] ^ rows[1]], 30), 30, 8)
    bad_pad = good[0][0].copy()
    bad_pad[0, -1] |= np.uint64(1 << 40)
    big = I.single_code("rand200x100")
    codes = good + [bad_rank, (bad_pad, good[0][1], good[0][2]), big]
    d, wits, st = B.md_batch(codes, B.md_options_init(work_budget=10 ** 11))
    assert st[:3] == [B.MD_OK] * 3
    assert st[3] == B.MD_ERANK and st[4] == B.MD_EINVAL and st[5] == B.MD_EBUDGET
    assert d[3] == d[4] == d[5] == -1
    # a stage limit leaves the code incomplete: best weight found so far, status MD_EBUDGET
    d2, w2, st2 = B.md_batch([big], B.md_options_init(max_stage=3))
    res = O.bz(big[0], big[1], big[2], stop_after_g=3)
    assert st2 == [B.MD_EBUDGET] and d2[0] == res.d and np.array_equal(w2[0], res.witness)


def test_batch_workload_sample(B):
    """The uneven batch workload (n in [48,160], k in [n/3, n/2]), first codes: batch vs single."""
    codes = [c for c in I.batch_codes(count=40) if c[1] <= 110]
    d, wits, st = B.md_batch(codes)
    assert all(s == B.MD_OK for s in st)
    for (G, n, k), di, wi in zip(codes, d, wits):
        ds, ws = single(B, G, n, k)
        assert di == ds and np.array_equal(wi, ws)


def test_batch_per_matrix_bound(B):
    codes = mixed_codes()
    d0, w0, s0 = B.md_batch(codes)
    d1, w1, s1 = B.md_batch(codes, B.md_options_init(stop_rule=1))
    assert s1 == [B.MD_OK] * len(codes) and d1 == d0
    assert all(np.array_equal(x, y) for x, y in zip(w0, w1))
    for (G, n, k), di, wi in zip(codes, d1, w1):
        res = O.bz(G, n, k, threads=8, stop_rule=1)
        assert di == res.d and np.array_equal(wi, res.witness)


@pytest.mark.parametrize("heavy", [1 << 12, 1 << 20, (1 << 64) - 1])
def test_batch_heavy_codes_run_alone(B, heavy):
    """Codes whose estimated work reaches batch_heavy run as single-code computations on two
    worker threads (tensor-core levels forced on, so the small codes here reach that kernel
    too) beside the shared schedule of the others; every result equals the oracle's,
    whichever route each code takes (2^12: most codes alone; 2^20: a mix; 2^64 - 1: none)."""
    codes = mixed_codes()
    d, wits, st = B.md_batch(codes, B.md_options_init(batch_heavy=heavy, tensor=2, tensor_head=3))
    assert st == [B.MD_OK] * len(codes)
    for (G, n, k), di, wi in zip(codes, d, wits):
        res = O.bz(G, n, k, threads=8)
        assert di == res.d and np.array_equal(wi, res.witness), (n, k, heavy)


def test_batch_workers_give_the_same_results(B):
    """The single-code runs give the same statuses, d and witnesses on one, two or four worker
    threads, and on the calling thread when a caller's allocator is set (the allocator is only
    ever called from that thread)."""
    import ctypes
    import threading
    torch = pytest.importorskip("torch")
    codes = mixed_codes()

    def same(a, b):
        return a[0] == b[0] and a[2] == b[2] and all(np.array_equal(x, y) for x, y in zip(a[1], b[1]))

    ref = B.md_batch(codes, B.md_options_init(batch_heavy=1 << 12, batch_workers=1))
    assert ref[2] == [B.MD_OK] * len(codes)
    for w in (2, 4):
        assert same(B.md_batch(codes, B.md_options_init(batch_heavy=1 << 12, batch_workers=w)), ref), w
    caller = threading.get_ident()
    seen, live = set(), {}

    def alloc(nbytes, ctx):
        seen.add(threading.get_ident())
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, ctx):
        live.pop(ptr, None)

    fa, ff = B.DEV_ALLOC(alloc), B.DEV_FREE(free)
    opt = B.md_options_init(batch_heavy=1 << 12, batch_workers=4)
    opt.dev_alloc = ctypes.cast(fa, ctypes.c_void_p)
    opt.dev_free = ctypes.cast(ff, ctypes.c_void_p)
    assert same(B.md_batch(codes, opt), ref)
    assert seen == {caller} and not live


def test_batch_tune_picks_cached_valid_options(B, tmp_path):
    """md_batch_tune times md_batch on samples of the batch, writes its choice to the JSON
    cache under the batch's key and the GPU's name, and reads it back on the next call without
    timing; md_batch with the tuned options (and with autotune = 1 through the cache) gives
    exactly the default options' results, which the oracle confirms on the small codes."""
    import json
    import time
    codes = I.batch_codes(count=256)
    base = B.md_options_init(work_budget=10 ** 9)
    cache = str(tmp_path / "tune.json")
    t0 = time.perf_counter()
    tuned = B.md_batch_tune(codes, base, cache)
    first = time.perf_counter() - t0
    assert tuned.chunk_log2 in (16, 18, 20) and tuned.blocks_per_sm in (0, 2, 4)
    assert tuned.batch_heavy in [1 << e for e in (30, 32, 34, 36, 38)]
    assert tuned.work_budget == 10 ** 9
    entries = json.load(open(cache))
    key = B.md_batch_tune_key(codes)
    (name, val), = entries.items()
    assert name.startswith(key + " | ")
    assert (val["chunk_log2"], val["blocks_per_sm"], val["batch_heavy"]) == \
        (tuned.chunk_log2, tuned.blocks_per_sm, tuned.batch_heavy)
    t0 = time.perf_counter()
    again = B.md_batch_tune(codes, base, cache)
    assert time.perf_counter() - t0 < first / 5
    assert (again.chunk_log2, again.blocks_per_sm, again.batch_heavy) == \
        (tuned.chunk_log2, tuned.blocks_per_sm, tuned.batch_heavy)
    ref = B.md_batch(codes, base)
    got = B.md_batch(codes, tuned)
    auto = B.md_batch(codes, B.md_options_init(work_budget=10 ** 9, autotune=1, tune_cache=cache.encode()))
    for r in (got, auto):
        assert r[0] == ref[0] and r[2] == ref[2]
        assert all(np.array_equal(x, y) for x, y in zip(r[1], ref[1]))
    checked = 0
    for (G, n, k), di, wi, si in zip(codes, *ref):
        if si == B.MD_OK and n <= 80:
            res = O.bz(G, n, k, threads=8)
            assert di == res.d and np.array_equal(wi, res.witness), (n, k)
            checked += 1
    assert checked >= 10
