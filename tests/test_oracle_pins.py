"""Pins of the CPU oracle to facts that do not come from the oracle itself.

- the paper's worked example of the colexicographic ("left-lexicographical") order and
  the printed lower-bound formula of Alg. 1 (tests/golden/);
- closed forms: binomial coefficients, C(k, g) combinations per level, textbook weight
  enumerators (Hamming, extended Golay, first-order Reed-Muller, simplex, repetition,
  single parity, trivial codes);
- brute force on small inputs, written in the test with itertools and Python integers;
- invariants: weight(witness) = d, witness in the row space, d <= n - k + 1, the
  structure of each Gamma_j (identity on its information set, reduced echelon form,
  same row space as G).
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from tests import textbook as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    return rows


# ------------------------------------------------------------------ colex order ---

def test_colex_paper_example():
    """Section 3.1: k=6, g=4, p=3 prefixes in left-lexicographical order."""
    expected = read_golden("colex_prefixes_k6_g4_p3.txt")
    k_eff = 6 - 1 - (4 - 3) + 1          # right-most element <= k-1-(g-p) = 4
    seq = [(0, 1, 2)]
    while True:
        nxt = O.colex_next(seq[-1], k_eff)
        if nxt is None:
            break
        seq.append(nxt)
    assert seq == expected
    assert len(seq) == math.comb(k_eff, 3) == 10      # task count C(k-(g-p), p)
    assert [O.colex_rank(c) for c in seq] == list(range(10))
    assert [O.colex_unrank(r, 3, k_eff) for r in range(10)] == expected


@pytest.mark.parametrize("k,g", [(1, 1), (5, 1), (5, 5), (7, 3), (9, 4), (12, 6), (10, 0)])
def test_colex_enumeration_is_complete(k, g):
    if g == 0:
        assert O.binomial(k, 0) == 1
        return
    c = tuple(range(g))
    seen = []
    while c is not None:
        seen.append(c)
        assert O.colex_rank(c) == T.colex_rank_formula(c) == len(seen) - 1
        assert O.colex_unrank(len(seen) - 1, g, k) == c
        c = O.colex_next(c, k)
    assert len(seen) == math.comb(k, g)
    assert sorted(seen) == list(itertools.combinations(range(k), g))


def test_colex_unrank_large():
    k, g = 100, 10
    rng = np.random.default_rng(7)
    for _ in range(50):
        c = tuple(sorted(rng.choice(k, size=g, replace=False).tolist()))
        r = T.colex_rank_formula(c)
        assert O.colex_rank(c) == r
        assert O.colex_unrank(r, g, k) == c
    with pytest.raises(O.OracleError):
        O.colex_unrank(math.comb(k, g), g, k)


def test_binomial_closed_form():
    for a in range(0, 70):
        for b in range(0, a + 2):
            assert O.binomial(a, b) == min(math.comb(a, b), (1 << 64) - 1), (a, b)
    assert O.binomial(200, 100) == (1 << 64) - 1      # saturates
    assert O.binomial(100, 13) == math.comb(100, 13)


# ----------------------------------------------------------------- brute force ---

@pytest.mark.parametrize("name", sorted(T.TEXTBOOK))
def test_bruteforce_textbook(name):
    ctor, d, counts = T.TEXTBOOK[name]
    rows, n, k = ctor()
    G = T.pack(rows, n)
    dmin, dist = O.bruteforce(G, n, k)
    assert dmin == d
    assert int(dist[0]) == 1
    assert int(dist.sum()) == 1 << k
    for w, cnt in counts.items():
        assert int(dist[w]) == cnt, (w, int(dist[w]), cnt)
    if name in ("hamming7", "golay24", "rm1_4", "simplex4", "repetition9", "trivial6"):
        # every weight class, against a Python enumeration of all codewords
        assert [int(x) for x in dist] == T.weight_distribution(rows, n)


def test_bruteforce_threads_and_rank_deficiency():
    """The message range split over 1, 2, 3, 5, 7 and 16 threads gives the whole weight
    distribution of a random [70,14] code, each time equal to a Python enumeration of all
    2^14 codewords (a range that overlaps, skips or shifts by one message shows up in it)."""
    rows = T.random_rows(70, 14, seed=3)
    G = T.pack(rows, 70)
    want = T.weight_distribution(rows, 70)
    assert sum(want) == 1 << 14
    for threads in (1, 2, 3, 5, 7, 16):
        d, dist = O.bruteforce(G, 70, 14, threads=threads)
        assert [int(x) for x in dist] == want, threads
        assert d == min(w for w in range(1, 71) if want[w])
    dup = T.pack(rows[:-1] + [rows[0]], 70)          # repeated row: rank 13
    d0, _ = O.bruteforce(dup, 70, 14)
    assert d0 == 0


# ------------------------------------------------------ info sets and Gamma_j ------

def check_gammas(rows, n, k):
    G = T.pack(rows, n)
    orders, ranks = O.info_sets(G, n, k)
    used = set()
    for j, (order, r) in enumerate(zip(orders, ranks)):
        assert sorted(order) == list(range(n))
        Gam, piv = O.gamma(G, n, k, order)
        assert piv == k
        grow = T.unpack(Gam)
        # same row space as G
        assert T.gf2_rank(rows + grow) == k and T.gf2_rank(grow) == k
        if r == k:
            S = order[:k]
            assert S == sorted(S) and not used.intersection(S)
            # the reduction order: the set's columns ascending, then every other column ascending
            assert order == S + [c for c in range(n) if c not in S]
            used.update(S)
            # identity on S_j, row i <-> i-th column of S_j
            for i in range(k):
                for t, c in enumerate(S):
                    assert (grow[i] >> c) & 1 == (1 if t == i else 0)
            # the columns of S_j are independent in G
            assert T.gf2_rank([T.column(rows, c) for c in S]) == k
        else:
            assert j == len(orders) - 1            # only the last set may be partial
            rest = [c for c in range(n) if c not in used]
            assert order == rest + sorted(used)
            assert T.gf2_rank([T.column(rows, c) for c in rest]) == r
        # reduced echelon form under `order`: leading entries advance, pivot columns unit
        lead = []
        for i in range(k):
            pos = next(p for p, c in enumerate(order) if (grow[i] >> c) & 1)
            lead.append(pos)
        assert lead == sorted(lead) and len(set(lead)) == k
        for i in range(k):
            col = order[lead[i]]
            assert sum((grow[t] >> col) & 1 for t in range(k)) == 1
        if r < k:
            # rows r..k-1 vanish on the set's columns: Gamma_m = [[I, A], [0, B]]
            for i in range(r, k):
                assert all(((grow[i] >> c) & 1) == 0 for c in order[:n - len(used)])
    # greedy: the sets are maximal while the leftover columns have rank < k
    assert len(used) + (0 if ranks[-1] == k else 0) <= n
    return orders, ranks


@pytest.mark.parametrize("n,k,seed", [(16, 5, 1), (24, 8, 2), (40, 13, 3), (70, 20, 4), (130, 40, 5),
                                      (64, 32, 6), (9, 9, 7), (33, 1, 8), (200, 100, 9)])
def test_gamma_structure(n, k, seed):
    rows = T.random_rows(n, k, seed)
    orders, ranks = check_gammas(rows, n, k)
    assert len(orders) >= 1


def test_info_sets_systematic_first_set_is_identity():
    from paper_1911_08963_gb300 import inputs
    G, n, k = inputs.single_code("rand128x64")
    orders, ranks = O.info_sets(G, n, k)
    assert ranks == [64, 64]
    assert orders[0][:64] == list(range(64))
    assert orders[1][:64] == list(range(64, 128))


def test_info_sets_leftover_rank_one_and_zero():
    """Section 2.1's disjoint information sets, as read here: after the full sets, all the
    leftover columns form the last set, of their own rank k_m, kept when k_m >= 1 and dropped
    when k_m = 0.  G = [I_4 | I_4 | e_0] has two identity sets and one leftover column of rank
    1; G = [I_4 | I_4 | 0] has an all-zero leftover column.  d = 2 for both (x = e_1 gives
    (e_1, e_1, 0)), as the brute force finds."""
    k, n = 4, 9
    for last, want_ranks in ((1, [4, 4, 1]), (0, [4, 4])):
        rows = [(1 << i) | (1 << (k + i)) | ((last << (2 * k)) if i == 0 else 0) for i in range(k)]
        G = T.pack(rows, n)
        orders, ranks = O.info_sets(G, n, k)
        assert ranks == want_ranks
        assert orders[0] == list(range(n)) and orders[1] == list(range(k, 2 * k)) + list(range(k)) + [2 * k]
        if last:
            assert orders[2] == [2 * k] + list(range(2 * k))
        check_gammas(rows, n, k)
        res = O.bz(G, n, k)
        assert res.d == O.bruteforce(G, n, k)[0] == 2
        assert res.m == len(want_ranks)


def test_bz_weight_one_codeword_stops_at_once():
    """Alg. 1 starts from L = 1 (every nonzero codeword has weight >= 1), so a weight-1
    codeword found in the first matrix at stage 1 ends the run before any other level:
    rows 0001 and 1110 (n = 4, k = 2) have the full set {0, 1}, a leftover set {2, 3} of
    rank 1, and d = 1 from row 0."""
    rows = [0b0001, 0b1110]
    G = T.pack(rows, 4)
    res = O.bz(G, 4, 2)
    assert res.d == 1 == O.bruteforce(G, 4, 2)[0]
    assert res.m == 2
    assert [lv[:2] for lv in res.levels] == [(1, 0)] and res.stop == (1, 0)


def test_rand64x32_bz_equals_the_definition():
    """At the [64,32] workload itself (seed 1), Alg. 1's d equals the definition's (Section
    2.1): the least weight over all 2^32 - 1 nonzero messages, by the multithreaded brute
    force, whose weight distribution covers all 2^32 codewords once.  The witness has that
    weight and lies in the row space."""
    from paper_1911_08963_gb300 import inputs
    G, n, k = inputs.single_code("rand64x32")
    d_bf, dist = O.bruteforce(G, n, k, threads=os.cpu_count() or 4)
    assert int(dist.sum()) == 1 << k and int(dist[0]) == 1
    res = O.bz(G, n, k)
    assert res.d == d_bf
    rows = T.unpack(G)
    wv = T.unpack(res.witness.reshape(1, -1))[0]
    assert T.wt(wv) == d_bf and T.solve_message(rows, wv) not in (None, 0)


def test_rank_errors():
    rows = T.random_rows(20, 6, 11)
    bad = T.pack(rows[:5] + [rows[0] ^ rows[1]], 20)
    with pytest.raises(O.OracleError):
        O.info_sets(bad, 20, 6)
    with pytest.raises(O.OracleError):
        O.bz(bad, 20, 6)
    assert O.rank(bad, 20, 6) == 5


# ---------------------------------------------------------- Brouwer-Zimmermann -----

def check_bz_invariants(rows, n, k, res):
    d = res.d
    wit = T.unpack(res.witness.reshape(1, -1))[0]
    assert 1 <= d <= n - k + 1                              # Singleton bound
    assert wit != 0 and T.wt(wit) == d
    msg = T.solve_message(rows, wit)
    assert msg is not None and msg != 0                     # witness = xG, x != 0
    assert res.L >= d or res.stop[0] == k                   # stopped by L >= U (or g = k)


@pytest.mark.parametrize("name", sorted(T.TEXTBOOK))
def test_bz_textbook(name):
    ctor, d, _ = T.TEXTBOOK[name]
    rows, n, k = ctor()
    for variant, rs in enumerate([rows, T.scramble(rows, n, 1), T.permute_columns(rows, n, 2)]):
        res = O.bz(T.pack(rs, n), n, k)
        assert res.d == d, (name, variant, res)
        check_bz_invariants(rs, n, k, res)


@pytest.mark.parametrize("n,k,seed", [(12, 4, 1), (20, 7, 2), (31, 10, 3), (48, 16, 4), (64, 18, 5),
                                      (66, 12, 6), (90, 15, 7), (150, 14, 8), (17, 16, 9), (25, 1, 10),
                                      (40, 20, 11), (57, 19, 12)])
def test_bz_matches_bruteforce(n, k, seed):
    rows = T.random_rows(n, k, seed)
    G = T.pack(rows, n)
    d_bf, dist = O.bruteforce(G, n, k)
    res = O.bz(G, n, k)
    assert res.d == d_bf
    check_bz_invariants(rows, n, k, res)
    res3 = O.bz(G, n, k, threads=3)
    assert (res3.d, res3.key, res3.levels) == (res.d, res.key, res.levels)


@pytest.mark.parametrize("n,k,seed", [(14, 5, 21), (22, 8, 22), (30, 10, 23), (36, 12, 24), (19, 9, 25),
                                      (26, 13, 26)])
def test_bz_levels_and_canonical_witness(n, k, seed):
    """Per-level (least weight, first colex rank) and the canonical witness, against an
    itertools enumeration of every level in (g, j) order."""
    rows = T.random_rows(n, k, seed)
    G = T.pack(rows, n)
    res = O.bz(G, n, k)
    gams, ranks, _ = O.gammas(G, n, k)
    grows = [T.unpack(x) for x in gams]
    U = None
    key = None
    for (g, j, w, first, count) in res.levels:
        assert count == math.comb(k, g)
        assert (w, first) == T.level_scan(grows[j], g)
        if U is None or w < U:
            U, key = w, (g, j, first)
    assert U == res.d and key == res.key
    # witness = sum of the rows of Gamma_j at the key's combination
    g, j, r = key
    c = O.colex_unrank(r, g, k)
    v = 0
    for i in c:
        v ^= grows[j][i]
    assert v == T.unpack(res.witness.reshape(1, -1))[0]
    # the canonical witness is the first weight-d codeword in (g, j, colex) order
    first_hit = None
    for (g2, j2, w2, f2, _) in res.levels:
        if w2 == res.d:
            first_hit = (g2, j2, f2)
            break
    assert first_hit == res.key


def test_bz_stop_rule_and_bound():
    """The run stops at the first check with L >= U; L follows Alg. 1's printed formula."""
    golden = read_golden("bz_bound_alg1.txt")
    for m, k, km, g, L in golden:
        ranks = [k] * (m - 1) + [km]
        assert sum(max(0, g + 1 - (k - r)) for r in ranks) == L
    for n, k, seed in [(30, 10, 31), (45, 12, 32), (64, 20, 33), (24, 11, 34)]:
        rows = T.random_rows(n, k, seed)
        G = T.pack(rows, n)
        res = O.bz(G, n, k)
        _, ranks = O.info_sets(G, n, k)
        m = len(ranks)
        # replay the stop rule on the level table
        L, U, stop_at = 1, None, None
        it = iter(res.levels)
        for g in range(1, k + 1):
            for j in range(m):
                rec = next(it)
                assert rec[:2] == (g, j)
                U = rec[2] if U is None else min(U, rec[2])
                if L >= U:
                    stop_at = (g, j)
                    break
            if stop_at:
                break
            if ranks[-1] < k:
                L = (m - 1) * (g + 1) + max(0, g + 1 - k + ranks[-1])
            else:
                L = m * (g + 1)
            if L >= U:
                stop_at = (g, m - 1)
                break
        assert stop_at == res.stop
        assert len(res.levels) == res.nlevels


@pytest.mark.parametrize("n,k,seed", [(12, 4, 1), (31, 10, 3), (48, 16, 4), (66, 12, 6), (40, 20, 11),
                                      (57, 19, 12), (30, 10, 31), (45, 12, 32)])
def test_bz_per_matrix_bound(n, k, seed):
    """Stop rule 1 (after matrix j of stage g: matrices <= j have completed stage g, the others
    stage g - 1) gives the same d and witness as Alg. 1 and brute force, runs a prefix of
    Alg. 1's levels, and stops exactly where the per-matrix bound first reaches U."""
    rows = T.random_rows(n, k, seed)
    G = T.pack(rows, n)
    a = O.bz(G, n, k)
    b = O.bz(G, n, k, stop_rule=1)
    d_bf, _ = O.bruteforce(G, n, k)
    assert b.d == a.d == d_bf
    assert b.key == a.key and np.array_equal(b.witness, a.witness)
    assert b.levels == a.levels[:len(b.levels)]
    check_bz_invariants(rows, n, k, b)
    _, ranks = O.info_sets(G, n, k)
    m = len(ranks)
    bound = lambda g, kj: max(0, g + 1 - (k - kj))
    U = None
    stop_at = None
    for rec in a.levels:
        g, j = rec[0], rec[1]
        U = rec[2] if U is None else min(U, rec[2])
        Lj = sum(bound(g if i <= j else g - 1, ranks[i]) for i in range(m))
        if Lj >= U:
            stop_at = (g, j)
            break
    assert stop_at == b.stop


def test_bz_partial_run_and_codeword_count():
    from paper_1911_08963_gb300 import inputs
    G, n, k = inputs.single_code("rand200x100")
    res = O.bz(G, n, k, threads=4, stop_after_g=2)
    assert [lv[:2] for lv in res.levels] == [(1, 0), (1, 1), (2, 0), (2, 1)]
    assert res.codewords == 2 * (100 + math.comb(100, 2))
    gams, ranks, _ = O.gammas(G, n, k)
    assert ranks == [100, 100]
    for g, j, w, first, count in res.levels:
        assert (w, first) == T.level_scan(T.unpack(gams[j]), g)


def test_scan_ranges_compose():
    rows = T.random_rows(60, 24, 41)
    G = T.pack(rows, 60)
    gams, _, _ = O.gammas(G, 60, 24)
    g = 4
    total = math.comb(24, g)
    whole = O.scan(gams[0], 60, 24, g, 0, total)
    parts = [O.scan(gams[0], 60, 24, g, a, min(total, a + 997)) for a in range(0, total, 997)]
    best = min(parts)          # (w, rank) lexicographic; ranges are disjoint
    assert best == whole
    assert O.scan(gams[0], 60, 24, g, 5, 5) == (61, (1 << 64) - 1)


def test_scan_range_past_the_level_is_clamped():
    """A rank range reaching past the level's C(k, g) combinations covers the level's end and
    no more: r1 beyond the end gives the same as r1 = C(k, g), and a range starting at or past
    the end is empty (weight n + 1, no rank)."""
    rows = T.random_rows(40, 12, 19)
    G = T.pack(rows, 40)
    gams, _, _ = O.gammas(G, 40, 12)
    for g in (1, 3, 6):
        total = math.comb(12, g)
        for r0 in (0, total // 2, total - 1):
            want = O.scan(gams[0], 40, 12, g, r0, total)
            for threads in (1, 3):
                assert O.scan(gams[0], 40, 12, g, r0, total + 5, threads=threads) == want
        assert O.scan(gams[0], 40, 12, g, total, total + 7) == (41, (1 << 64) - 1)


def test_scan_subranges_and_threads_against_enumeration():
    """The scan of any colex-rank range [r0, r1), split over 1, 2, 3, 5 or 7 threads, returns
    the least weight in that range and its first rank, as a Python enumeration of the same
    g-subsets in colex order (tuples sorted by their reversed elements) finds them.  Small
    ranges, ranges ending right after a level minimum, and whole levels are included, so a
    split that drops, repeats or shifts a rank, or a tie resolved to a later thread, fails."""
    n, k = 40, 14
    rows = T.random_rows(n, k, 77)
    G = T.pack(rows, n)
    gams, _, _ = O.gammas(G, n, k)
    grow = T.unpack(gams[0])
    rng = np.random.default_rng(5)
    for g in (1, 2, 3, 5):
        combos = sorted(itertools.combinations(range(k), g), key=lambda c: c[::-1])
        weights = []
        for c in combos:
            v = 0
            for i in c:
                v ^= grow[i]
            weights.append(T.wt(v))
        total = len(combos)
        wmin = min(weights)
        last_min = max(r for r, w in enumerate(weights) if w == wmin)
        ranges = [(0, total), (0, last_min + 1), (last_min, total), (last_min, last_min + 1)]
        for _ in range(12):
            a, b = sorted(int(x) for x in rng.integers(0, total + 1, size=2))
            if a < b:
                ranges.append((a, b))
        for r0, r1 in ranges:
            w = min(weights[r0:r1])
            want = (w, r0 + weights[r0:r1].index(w))
            for threads in (1, 2, 3, 5, 7):
                assert O.scan(gams[0], n, k, g, r0, r1, threads=threads) == want, (g, r0, r1, threads)
