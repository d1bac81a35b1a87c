"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Compared on the same seeded inputs: d, the canonical witness, its key (g, j, colex rank),
and every per-level record (least weight and first colex rank reaching it; the kernels
resolve a level's least weight only up to the bound U held before the level, so the
oracle's record is reported as -1 where it exceeds that bound).  All results are integers:
the tolerance is zero.
"""
import math
import os

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


def expected_levels(res, n):
    out = []
    U = n + 1
    for g, j, w, first, count in res.levels:
        out.append((g, j, w, first, count) if w <= U else (g, j, -1, 0, count))
        U = min(U, w)
    return out


def run_gpu(B, G, n, k, **opts):
    opt = B.md_options_init(**opts)
    h = B.md_create(G, n, k, opt)
    try:
        d, wit = B.md_compute(h, n)
        return d, wit, B.md_info_get(h), B.md_levels(h)
    finally:
        B.md_destroy(h)


def assert_parity(B, G, n, k, res=None, threads=1, **opts):
    if res is None:
        res = O.bz(G, n, k, threads=threads)
    d, wit, info, levels = run_gpu(B, G, n, k, **opts)
    assert d == res.d
    assert np.array_equal(wit, res.witness)
    assert (info["key_g"], info["key_j"], info["key_rank"]) == res.key
    assert levels == expected_levels(res, n)
    assert info["complete"] == 1
    assert info["codewords"] == res.codewords
    assert (info["stop_g"], info["stop_j"]) == res.stop
    assert info["lower_bound"] == res.L
    return res, info


@pytest.mark.parametrize("name", sorted(T.TEXTBOOK))
def test_textbook_codes(B, name):
    ctor, d, _ = T.TEXTBOOK[name]
    rows, n, k = ctor()
    for rs in (rows, T.scramble(rows, n, 5), T.permute_columns(rows, n, 6)):
        res, info = assert_parity(B, T.pack(rs, n), n, k)
        assert res.d == d


RANDOM_CASES = [(8, 3, 1), (20, 7, 2), (31, 10, 3), (48, 16, 4), (64, 18, 5), (66, 12, 6), (90, 15, 7),
                (150, 14, 8), (17, 16, 9), (25, 1, 10), (40, 20, 11), (57, 19, 12), (100, 33, 13),
                (120, 40, 14), (96, 44, 15), (100, 40, 16), (130, 30, 17), (70, 35, 18), (80, 38, 19),
                (90, 45, 20), (126, 42, 21)]
_ORACLE_CACHE = {}


def oracle_bz_cached(G, n, k, key):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = O.bz(G, n, k, threads=THREADS)
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("n,k,seed", RANDOM_CASES)
@pytest.mark.parametrize("filt", [0, 1, 2, 3])
def test_random_codes(B, n, k, seed, filt):
    rows = T.random_rows(n, k, seed)
    G = T.pack(rows, n)
    res = oracle_bz_cached(G, n, k, (n, k, seed))
    assert_parity(B, G, n, k, res=res, filter=filt)


def test_small_chunks_and_block_shapes(B):
    """Tiny work items and unusual launch shapes cover many item boundaries and ragged tails."""
    rows = T.random_rows(90, 30, 77)
    G = T.pack(rows, 90)
    res = O.bz(G, 90, 30, threads=THREADS)
    for opts in (dict(chunk_log2=8), dict(chunk_log2=12, threads_per_block=96), dict(blocks_per_sm=1),
                 dict(threads_per_block=32, chunk_log2=10)):
        assert_parity(B, G, 90, 30, res=res, **opts)


def test_rand64x32(B):
    G, n, k = I.single_code("rand64x32")
    res, info = assert_parity(B, G, n, k)
    d_bf, dist = O.bruteforce(G, n, k, threads=THREADS)
    assert res.d == d_bf


def test_rand128x64(B):
    G, n, k = I.single_code("rand128x64")
    res = O.bz(G, n, k, threads=THREADS)
    assert_parity(B, G, n, k, res=res)
    assert_parity(B, G, n, k, res=res, filter=0)


def test_rand200x100_first_stages(B):
    """[200,100]: every level of stages 1..5 (about 1.6e8 combinations) against the oracle."""
    G, n, k = I.single_code("rand200x100")
    res = O.bz(G, n, k, threads=THREADS, stop_after_g=5)
    d, wit, info, levels = run_gpu(B, G, n, k, max_stage=5)
    assert levels == expected_levels(res, n)
    assert d == res.d and np.array_equal(wit, res.witness)
    assert info["complete"] == 0


def task_ranges(k, g, M, u0, u1):
    """Colex rank ranges of the combinations of md_scan_task(g, M, [u0, u1))."""
    P = 2 if g == 5 else 3
    v = g - P - 1
    heads = math.comb(M, P)
    out = []
    for u in range(u0, u1):
        up = O.colex_unrank(u, v, k - 1 - M)
        rhi = math.comb(M, P + 1) + sum(math.comb(M + 1 + e, P + 2 + t) for t, e in enumerate(up))
        out.append((rhi, rhi + heads))
    return out


def oracle_task(gam, n, k, g, M, u0, u1, bound=-1):
    best = (n + 1, 0)
    for r0, r1 in task_ranges(k, g, M, u0, u1):
        best = min(best, O.scan(gam, n, k, g, r0, r1, threads=THREADS))
    if bound >= 0 and best[0] > bound:
        return (-1, 0)
    return best


@pytest.mark.parametrize("g", [6, 9, 10])
def test_rand200x100_sampled_tasks(B, g):
    """Full-size [200,100] levels, sampled: tasks of the production kernel against the oracle."""
    G, n, k = I.single_code("rand200x100")
    gams, _, _ = O.gammas(G, n, k)
    rng = np.random.default_rng(1000 + g)
    h = B.md_create(G, n, k)
    try:
        for j in (0, 1):
            for _ in range(3):
                M = int(rng.integers(8, 40))
                nup = math.comb(k - 1 - M, g - 4)
                u0 = int(rng.integers(0, nup - 64))
                u1 = u0 + int(rng.integers(1, 64))
                for bound in (-1, 30, 0):
                    got = B.md_scan_task(h, g, j, M, u0, u1, bound)
                    assert got == oracle_task(gams[j], n, k, g, M, u0, u1, bound), (g, j, M, u0, u1, bound)
    finally:
        B.md_destroy(h)


def oracle_range(gam, n, k, g, r0, r1):
    """Oracle scan of a rank range; an empty range reports (-1, 0) like the library."""
    w, r = O.scan(gam, n, k, g, r0, r1, threads=THREADS)
    return (w, r) if w <= n else (-1, 0)


def test_rand200x100_sampled_ranges(B):
    G, n, k = I.single_code("rand200x100")
    gams, _, _ = O.gammas(G, n, k)
    rng = np.random.default_rng(7)
    h = B.md_create(G, n, k)
    try:
        for g in (3, 7, 10):
            total = math.comb(k, g)
            for j in (0, 1):
                span = min(300000, total // 2)
                r0 = int(rng.integers(0, total - span))
                r1 = r0 + int(rng.integers(1, span))
                assert B.md_scan_range(h, g, j, r0, r1) == oracle_range(gams[j], n, k, g, r0, r1)
        assert B.md_scan_range(h, 4, 0, 10, 10) == (-1, 0)
    finally:
        B.md_destroy(h)


def test_scan_range_matches_oracle_small(B):
    rows = T.random_rows(75, 22, 31)
    G = T.pack(rows, 75)
    gams, _, _ = O.gammas(G, 75, 22)
    h = B.md_create(G, 75, 22)
    try:
        rng = np.random.default_rng(3)
        for g in (1, 2, 5, 8):
            total = math.comb(22, g)
            for _ in range(4):
                r0 = int(rng.integers(0, total))
                r1 = int(rng.integers(r0, total + 1))
                for j in range(len(gams)):
                    assert B.md_scan_range(h, g, j, r0, r1) == oracle_range(gams[j], 75, 22, g, r0, r1)
            # the whole level equals the oracle's level scan
            assert B.md_scan_range(h, g, 0, 0, total) == oracle_range(gams[0], 75, 22, g, 0, total)
            for bound in (0, 20, 40):
                want = oracle_range(gams[0], 75, 22, g, 0, total)
                want = want if want[0] <= bound else (-1, 0)
                assert B.md_scan_range(h, g, 0, 0, total, bound) == want
    finally:
        B.md_destroy(h)


def test_wide_rows_and_global_pair_table(B):
    """n = 256 with a rank-deficient last Gamma (all 256 columns packed, 8 words) and a pair
    table too large for shared memory (k = 150)."""
    rows = T.random_rows(256, 150, 41)
    G = T.pack(rows, 256)
    gams, ranks, _ = O.gammas(G, 256, 150)
    assert ranks[0] == 150 and ranks[-1] < 150
    h = B.md_create(G, 256, 150)
    try:
        jlast = len(gams) - 1
        for g, M, u0, u1 in ((6, 20, 5, 40), (5, 30, 0, 30)):
            for j in (0, jlast):
                assert B.md_scan_task(h, g, j, M, u0, u1) == oracle_task(gams[j], 256, 150, g, M, u0, u1)
        total = math.comb(150, 3)
        assert B.md_scan_range(h, 3, jlast, 0, total) == O.scan(gams[jlast], 256, 150, 3, 0, total, threads=THREADS)
    finally:
        B.md_destroy(h)


@pytest.mark.parametrize("n,k,seed", [(1, 1, 0), (5, 5, 1), (12, 1, 2), (256, 3, 3), (256, 250, 4), (200, 195, 5),
                                      (129, 64, 6), (65, 2, 7)])
def test_edge_shapes(B, n, k, seed):
    rows = T.random_rows(n, k, seed) if n > 1 else [1]
    assert_parity(B, T.pack(rows, n), n, k, threads=THREADS)


def test_repeat_and_interleaved_handles(B):
    a = T.random_rows(60, 20, 51)
    b = T.random_rows(80, 30, 52)
    Ga, Gb = T.pack(a, 60), T.pack(b, 80)
    ha, hb = B.md_create(Ga, 60, 20), B.md_create(Gb, 80, 30)
    try:
        r1 = B.md_compute(ha, 60)
        s1 = B.md_compute(hb, 80)
        r2 = B.md_compute(ha, 60)
        s2 = B.md_compute(hb, 80)
        assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1])
        assert s1[0] == s2[0] and np.array_equal(s1[1], s2[1])
        assert r1[0] == O.bz(Ga, 60, 20).d and s1[0] == O.bz(Gb, 80, 30).d
    finally:
        B.md_destroy(ha)
        B.md_destroy(hb)


def test_budget_and_max_stage(B):
    G, n, k = I.single_code("rand128x64")
    opt = B.md_options_init(work_budget=10 ** 6)
    h = B.md_create(G, n, k, opt)
    try:
        with pytest.raises(B.MDError) as e:
            B.md_compute(h, n)
        assert e.value.code == B.MD_EBUDGET
    finally:
        B.md_destroy(h)
    d, wit, info, levels = run_gpu(B, G, n, k, max_stage=3)
    res = O.bz(G, n, k, stop_after_g=3)
    assert info["complete"] == 0 and d == res.d and levels == expected_levels(res, n)


@pytest.mark.parametrize("n,k,seed", [(80, 40, 121), (96, 48, 145), (96, 48, 154)])
def test_mid_level_stop(B, n, k, seed):
    """Codes whose minimum weight equals the lower bound of the previous stage and first
    appears in the middle of a split level: once U <= L the kernel skips work ranked after
    the level's best codeword.  Every record still equals the oracle's."""
    G = I.random_code(n, k, seed)
    res = O.bz(G, n, k, threads=THREADS)
    _, info = assert_parity(B, G, n, k, res=res)
    # with one warp per SM the level's work items run in many waves, so work handed out after
    # the settling codeword is found is skipped
    _, slow = assert_parity(B, G, n, k, res=res, threads_per_block=32, blocks_per_sm=1)
    SKIPPED.append(slow["skipped_work"])


SKIPPED = []


def test_mid_level_stop_skipped_work():
    """The skip happened for at least one of the codes above (timing-dependent per code)."""
    assert SKIPPED and max(SKIPPED) > 0


@pytest.mark.parametrize("n,k,seed", RANDOM_CASES)
def test_random_codes_per_matrix_bound(B, n, k, seed):
    """Stop rule 1 (per-matrix bound) against the oracle with the same rule: same levels,
    stop and witness; d and witness also equal the Alg. 1 run's."""
    rows = T.random_rows(n, k, seed)
    G = T.pack(rows, n)
    res = O.bz(G, n, k, threads=THREADS, stop_rule=1)
    base = oracle_bz_cached(G, n, k, (n, k, seed))
    assert (res.d, res.key) == (base.d, base.key)
    assert_parity(B, G, n, k, res=res, stop_rule=1)


@pytest.mark.parametrize("n,k,seed", [(64, 32, 1), (90, 40, 3), (48, 16, 5), (100, 33, 13)])
def test_permuted_column_order(B, n, k, seed):
    """perm_trials: the run on the chosen column order equals the oracle's run on the
    permuted matrix, with the witness mapped back to the caller's columns; d is unchanged."""
    from tests.test_perm_search import choose_order, permute, to_caller
    G = I.random_code(n, k, seed) if seed != 13 else T.pack(T.random_rows(n, k, seed), n)
    order, _ = choose_order(G, n, k, 12, 99 + seed)
    res = O.bz(permute(G, n, k, order), n, k, threads=THREADS)
    d, wit, info, levels = run_gpu(B, G, n, k, perm_trials=12, perm_seed=99 + seed)
    assert d == res.d == O.bz(G, n, k, threads=THREADS).d
    assert T.unpack(wit.reshape(1, -1)) == to_caller(T.unpack(res.witness.reshape(1, -1)), order, n)
    assert (info["key_g"], info["key_j"], info["key_rank"]) == res.key
    assert levels == expected_levels(res, n)
