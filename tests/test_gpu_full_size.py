"""GPU: the complete minimum-distance computation of the random [200,100] code (seed 3), the
workload the throughput and time-to-d figures are quoted on.

The whole run (about 3.2e14 combinations, stages 1..11) is far beyond the oracle, so the
result is pinned by what the definition and Alg. 1 fix at any size:
  * the run is complete: the lower bound L(g) = sum_j max(0, g + 1 - (k - k_j)) of the last
    stage reached U (Alg. 1's stopping rule), and L >= d;
  * the witness is a nonzero codeword (it is xG for a message x, solved over F2 here with
    the tests' own elimination) whose weight, counted here, is d (Section 2.1's definition
    of d as the least weight of a nonzero codeword, reached by it);
  * the witness key (g, j, colex rank) reproduces the witness: the rows of Gamma_j at the
    unranked combination XOR to it;
  * the CPU oracle scans the 2^23 colex ranks of level (g, j) that end at the key one by one
    and returns exactly (d, key rank): no lighter codeword, and none of weight d ranked
    earlier, in that window;
  * every level record is either absent or at least d, and the first level with a record
    of weight d is the key's level.
A slow companion runs the same computation on the popcount kernels alone (no tensor cores)
and requires identical d, witness, key and level records.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_08963_gb300 import inputs as I
from tests import textbook as T

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
WINDOW = 1 << 23


@pytest.fixture(scope="module")
def B():
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding
    return binding


def full_run(B, **opts):
    G, n, k = I.single_code("rand200x100")
    h = B.md_create(G, n, k, B.md_options_init(**opts))
    try:
        d, wit = B.md_compute(h, n)
        info = B.md_info_get(h)
        levels = B.md_levels(h)
        gam = [B.md_gamma(h, j, n, k)[0] for j in range(info["m"])]
    finally:
        B.md_destroy(h)
    return d, wit, info, levels, gam


@pytest.fixture(scope="module")
def default_run(B):
    return full_run(B)


def test_full_rand200x100_to_d(B, default_run):
    G, n, k = I.single_code("rand200x100")
    d, wit, info, levels, gam = default_run
    assert info["complete"] == 1
    assert info["lower_bound"] >= d
    assert d <= n - k + 1                                  # Singleton bound
    # the last stage's bound is Alg. 1's: two full-rank information sets give L = 2 (g + 1)
    assert info["m"] == 2 and info["ranks"][:2] == [k, k]
    assert info["lower_bound"] == 2 * (info["stop_g"] + 1)
    # the witness: weight d by our own count, nonzero, in the row space of G
    wv = T.unpack(wit[None, :])[0]
    assert wv != 0 and T.wt(wv) == d
    x = T.solve_message(T.unpack(G), wv)
    assert x is not None and x != 0
    # the key reproduces the witness
    kg, kj, kr = info["key_g"], info["key_j"], info["key_rank"]
    comb = O.colex_unrank(kr, kg, k)
    row = np.zeros(gam[kj].shape[1], dtype=np.uint64)
    for c in comb:
        row ^= gam[kj][c]
    assert np.array_equal(row, wit)
    # the oracle's scan of the window ending at the key: exactly (d, key rank)
    gams, _, _ = O.gammas(G, n, k)
    assert np.array_equal(gams[kj], gam[kj])
    r0 = max(0, kr + 1 - WINDOW)
    assert O.scan(gams[kj], n, k, kg, r0, kr + 1, threads=THREADS) == (d, kr)
    # level records: none lighter than d, the key's level is the first reaching d
    first_d = None
    for idx, (g, j, w, first, count) in enumerate(levels):
        assert w == -1 or w >= d, (g, j, w)
        if w == d and first_d is None:
            first_d = (g, j, first)
    assert first_d == (kg, kj, kr)
    assert (levels[-1][0], levels[-1][1]) == (info["stop_g"], info["stop_j"])


def test_full_rand200x100_records_have_their_weight(B, default_run):
    """Each level record's combination (rows of Gamma_j at its colex rank) has the recorded
    weight, counted here."""
    _, _, info, levels, gam = default_run
    k = info["k"]
    for g, j, w, first, _ in levels:
        if w < 0:
            continue
        row = np.zeros(gam[j].shape[1], dtype=np.uint64)
        for c in O.colex_unrank(first, g, k):
            row ^= gam[j][c]
        assert sum(bin(int(v)).count("1") for v in row) == w, (g, j)


@pytest.mark.slow
def test_full_rand200x100_popcount_kernels_agree(B, default_run):
    """The same computation with the tensor cores off (popcount kernels for every level)."""
    d, wit, info, levels, _ = default_run
    d0, wit0, info0, levels0, _ = full_run(B, tensor=0)
    assert d0 == d and np.array_equal(wit0, wit)
    assert (info0["key_g"], info0["key_j"], info0["key_rank"]) == (info["key_g"], info["key_j"], info["key_rank"])
    assert levels0 == levels
    assert info0["complete"] == 1 and info0["lower_bound"] == info["lower_bound"]


def test_full_rand200x100_stage11_windows_hold_nothing_lighter(B, default_run):
    """Stage 11 is where d is first reached and proven (L = 2 * 12 = 24).  The oracle scans
    spread colex windows of 2^22 ranks in both of its levels (the first ranks, the last, and
    six at seeded random offsets): no window holds a codeword lighter than d, and a window
    holding a codeword of weight d belongs to a level whose record has weight d and a rank no
    later than the window's first rank of that weight (the record is the level's first rank of its least
    weight, and d is at most the U held before either level)."""
    import math
    G, n, k = I.single_code("rand200x100")
    d, _, info, levels, gam = default_run
    gams, _, _ = O.gammas(G, n, k)
    rng = np.random.default_rng(11)
    win = 1 << 22
    total = math.comb(k, 11)
    recs = {(g, j): (w, first) for g, j, w, first, _ in levels}
    assert (11, 0) in recs and (11, 1) in recs
    for j in (0, 1):
        assert np.array_equal(gams[j], gam[j])
        w_rec, first_rec = recs[(11, j)]
        starts = [0, total - win] + [int(x) for x in rng.integers(0, total - win, size=6)]
        for r0 in starts:
            w, first = O.scan(gams[j], n, k, 11, r0, r0 + win, threads=THREADS)
            assert w >= d, (j, r0, w)
            if w == d:
                # weight d is at most the U held before either level, so the level records it
                assert w_rec == d and first >= first_rec, (j, r0, first, w_rec, first_rec)
