"""GPU parity of the tensor-core levels (md_options.tensor) against the CPU oracle.

tensor = 2 runs every level with g >= q + 1 through the tcgen05 kernel, whatever its size, so
small codes cover: head sizes q = 2 and 3, every packed row width W = 1..8 (one MMA per 32
packed bits), partial head slices (C(s, q) not a multiple of 256), ragged tail runs, tails
with no upper elements (g = q + 1), rank-deficient last matrices (base 0) and both stop rules.
Every comparison is exact: d, witness, key and every per-level record.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_08963_gb300 import inputs as I
from tests import textbook as T

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
_CACHE = {}


@pytest.fixture(scope="module")
def B():
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding
    return binding


def oracle_cached(G, n, k, key, **kw):
    kk = (key, tuple(sorted(kw.items())))
    if kk not in _CACHE:
        _CACHE[kk] = O.bz(G, n, k, threads=THREADS, **kw)
    return _CACHE[kk]


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


def assert_parity(B, G, n, k, res, **opts):
    d, wit, info, levels = run_gpu(B, G, n, k, **opts)
    assert d == res.d
    assert np.array_equal(wit, res.witness)
    assert (info["key_g"], info["key_j"], info["key_rank"]) == res.key
    assert levels == expected_levels(res, n)
    assert (info["stop_g"], info["stop_j"]) == res.stop
    assert info["lower_bound"] == res.L
    return info


# (n, k, seed): packed widths W = ceil((n - k) / 32) from 1 to 8, and codes whose last
# information set is rank-deficient (every column packed, weight base 0)
CASES = [(40, 12, 31), (64, 24, 32), (90, 30, 33), (120, 40, 34), (160, 24, 35), (200, 24, 36),
         (224, 28, 37), (256, 20, 38), (150, 14, 39), (70, 35, 40), (100, 33, 41), (57, 19, 42)]


@pytest.mark.parametrize("n,k,seed", CASES)
@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_forced_tensor_levels(B, n, k, seed, q):
    G = T.pack(T.random_rows(n, k, seed), n)
    res = oracle_cached(G, n, k, (n, k, seed))
    assert_parity(B, G, n, k, res, tensor=2, tensor_head=q)


@pytest.mark.parametrize("n,k,seed", CASES)
@pytest.mark.parametrize("filt", [0, 3])
def test_forced_tensor_product_words(B, n, k, seed, filt):
    """The product's word count: filter = 0 always multiplies every packed word (the product is
    the exact weight); filter = 3 always multiplies the first word only, so the product is a
    lower bound and nearly every row goes through the exact recheck of its candidate columns
    (tail sum XOR head sum over all words).  Both must give exactly the oracle's results."""
    G = T.pack(T.random_rows(n, k, seed), n)
    res = oracle_cached(G, n, k, (n, k, seed))
    assert_parity(B, G, n, k, res, tensor=2, tensor_head=3, filter=filt)


@pytest.mark.parametrize("n,k,seed", [(90, 30, 33), (100, 33, 41), (120, 40, 34)])
def test_forced_tensor_per_matrix_rule(B, n, k, seed):
    G = T.pack(T.random_rows(n, k, seed), n)
    res = oracle_cached(G, n, k, (n, k, seed), stop_rule=1)
    assert_parity(B, G, n, k, res, tensor=2, tensor_head=3, stop_rule=1)


@pytest.mark.parametrize("name", sorted(T.TEXTBOOK))
def test_forced_tensor_textbook(B, name):
    ctor, d, _ = T.TEXTBOOK[name]
    rows, n, k = ctor()
    G = T.pack(rows, n)
    res = O.bz(G, n, k, threads=THREADS)
    assert_parity(B, G, n, k, res, tensor=2, tensor_head=3)
    assert res.d == d


def test_rand128x64_tensor(B):
    """[128, 64]: stages 7.. are tensor-core levels by default (C(64, g) >= 2^28)."""
    G, n, k = I.single_code("rand128x64")
    res = oracle_cached(G, n, k, "rand128x64")
    info = assert_parity(B, G, n, k, res)
    assert info["complete"] == 1
    assert_parity(B, G, n, k, res, tensor=2, tensor_head=2)


def test_rand200x100_stage6_tensor(B):
    """[200, 100] up to stage 6: the g = 6 levels (C(100, 6) = 1.2e9 each) run on the tensor
    cores by default (q = 3, tails of one pivot and two upper elements)."""
    G, n, k = I.single_code("rand200x100")
    res = O.bz(G, n, k, threads=THREADS, stop_after_g=6)
    d, wit, info, levels = run_gpu(B, G, n, k, max_stage=6)
    assert levels == expected_levels(res, n)
    assert d == res.d


def test_tensor_matches_split_kernel_stage10(B):
    """Consistency at the benchmark's configuration ([200,100] seed 3, stages g <= 10, the
    launches bench.py times), beyond the oracle's reach for whole levels: the records of the
    tensor-core levels g = 6..10 equal those of the popcount kernels (themselves pinned to
    the oracle by sampled tasks), and each record's codeword has the recorded weight."""
    G, n, k = I.single_code("rand200x100")
    _, _, _, lev_tc = run_gpu(B, G, n, k, max_stage=10, tensor=1)
    _, _, _, lev_pc = run_gpu(B, G, n, k, max_stage=10, tensor=0)
    assert lev_tc == lev_pc
    assert max(lv[0] for lv in lev_tc) == 10
    opt = B.md_options_init()
    h = B.md_create(G, n, k, opt)
    try:
        gam = [B.md_gamma(h, j, n, k)[0] for j in range(2)]
    finally:
        B.md_destroy(h)
    for g, j, w, first, _ in lev_tc:
        if w < 0:
            continue
        comb = O.colex_unrank(first, g, k)
        row = np.zeros(gam[j].shape[1], dtype=np.uint64)
        for c in comb:
            row ^= gam[j][c]
        assert sum(bin(int(x)).count("1") for x in row) == w


@pytest.mark.parametrize("n,k,gmax,seed", [(256, 60, 8, 51), (256, 100, 7, 52), (230, 40, 9, 53), (240, 80, 7, 54)])
def test_tensor_wide_rows_production_levels(B, n, k, gmax, seed):
    """Wide packed rows at production level sizes (the default rule picks the tensor cores for
    C(k, g) >= 2^28): W = 5..7, so tile sets of T = 2 and T = 1 tiles, up to five matrices
    with a rank-deficient last one.  The records equal those of the popcount kernels, each
    record's codeword (rows of Gamma_j at the record's colex rank) has the recorded weight,
    and the oracle's scan of the 2^22 colex ranks ending at each record returns exactly the
    record (no lighter codeword there, and none of its weight ranked earlier)."""
    import math
    G = T.pack(T.random_rows(n, k, seed), n)
    _, _, _, lev_tc = run_gpu(B, G, n, k, max_stage=gmax, tensor=1)
    _, _, _, lev_pc = run_gpu(B, G, n, k, max_stage=gmax, tensor=0)
    assert lev_tc == lev_pc
    assert any(math.comb(k, lv[0]) >= 1 << 28 for lv in lev_tc)
    gams, _, _ = O.gammas(G, n, k)
    h = B.md_create(G, n, k, B.md_options_init())
    try:
        gam = {}
        for g, j, w, first, _ in lev_tc:
            if w < 0:
                continue
            if j not in gam:
                gam[j] = B.md_gamma(h, j, n, k)[0]
                assert np.array_equal(gams[j], gam[j]), j
            row = np.zeros(gam[j].shape[1], dtype=np.uint64)
            for c in O.colex_unrank(first, g, k):
                row ^= gam[j][c]
            assert sum(bin(int(x)).count("1") for x in row) == w, (g, j)
            r0 = max(0, first + 1 - (1 << 22))
            assert O.scan(gams[j], n, k, g, r0, first + 1, threads=THREADS) == (w, first), (g, j)
    finally:
        B.md_destroy(h)


def test_tensor_stage10_record_is_window_minimum(B):
    """Sampled outputs at full size: for each level (10, j) the oracle scans colex-rank
    windows one combination at a time (the first ranks, ranks ending at the record, and
    windows spread over the level); no codeword there is lighter than the level's record,
    and the record's own rank has the recorded weight."""
    import math
    G, n, k = I.single_code("rand200x100")
    gams, _, _ = O.gammas(G, n, k)
    d, _, _, levels = run_gpu(B, G, n, k, max_stage=10)
    total = math.comb(k, 10)
    span = 1 << 23
    checked = 0
    for g, j, w, first, count in levels:
        if g != 10:
            continue
        checked += 1
        starts = [0] + [(total // 5) * i for i in range(1, 5)]
        if w >= 0:
            starts.append(max(0, first + 1 - span))
        for r0 in starts:
            r1 = min(total, r0 + span)
            wmin, rmin = O.scan(gams[j], n, k, g, r0, r1, threads=THREADS)
            # no record: the whole level is heavier than the bound held before it (>= d)
            assert wmin >= w if w >= 0 else wmin > d, (j, r0)
            if w >= 0 and r0 <= first < r1:
                assert (wmin, rmin) == (w, first), (j, r0)
    assert checked == 2


def test_tensor_mid_level_stop(B):
    """The tensor-core scheduler skips work items ranked above the settled record once U <= L;
    the result stays exact."""
    G = T.pack(T.random_rows(100, 33, 41), 100)
    res = oracle_cached(G, 100, 33, (100, 33, 41))
    info = assert_parity(B, G, 100, 33, res, tensor=2, tensor_head=3)
    assert info["skipped_work"] >= 0


def test_tensor_wait_timeout_is_reported(B):
    """Failure detection without a fault: with the test hook set, the tail producers never
    signal their first tile set, every block's bounded wait runs out (4 s), frees its tensor
    memory and returns, the run stops, and md_compute reports MD_ETIMEOUT; the context stays
    usable and the next run is exact."""
    G, n, k = I.single_code("rand64x32")
    res = oracle_cached(G, n, k, "rand64x32")
    h = B.md_create(G, n, k, B.md_options_init(tensor=2, tensor_head=3, test_stall=1))
    try:
        with pytest.raises(B.MDError) as e:
            B.md_compute(h, n)
        assert e.value.code == 8                       # MD_ETIMEOUT
    finally:
        B.md_destroy(h)
    assert_parity(B, G, n, k, res, tensor=2, tensor_head=3)
