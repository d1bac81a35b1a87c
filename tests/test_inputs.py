"""The seeded input generators: published SplitMix64 outputs, packing, workload shapes."""
import math

import numpy as np

import oracle as O
from paper_1911_08963_gb300 import inputs as I
from tests import textbook as T


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 seeded with 0 (the reference implementation's test vector)
    r = I.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_systematic_packing():
    for n, k, seed in [(64, 32, 1), (128, 64, 2), (200, 100, 3), (65, 20, 9), (48, 24, 4)]:
        G = I.random_code(n, k, seed)
        assert G.shape == (k, (n + 63) // 64) and G.dtype == np.uint64
        rows = T.unpack(G)
        for i, r in enumerate(rows):
            assert r >> n == 0                       # padding bits are zero
            assert r & ((1 << k) - 1) == 1 << i      # identity block
        # R is roughly balanced
        ones = sum(T.wt(r >> k) for r in rows)
        assert abs(ones / (k * (n - k)) - 0.5) < 0.08


def test_single_codes_use_first_invertible_draw():
    for name, c in I.SINGLE.items():
        n, k, seed = c["n"], c["k"], c["seed"]
        for skip in range(c["skip"]):
            _, ranks = O.info_sets(I.random_code(n, k, seed, skip), n, k)
            assert ranks != [k, k]
        G, n2, k2 = I.single_code(name)
        assert (n2, k2) == (n, k)
        _, ranks = O.info_sets(G, n, k)
        assert ranks == [k, k]


def test_batch_shapes():
    codes = I.batch_codes(count=300)
    assert len(codes) == 300
    for G, n, k in codes:
        assert 48 <= n <= 160 and math.ceil(n / 3) <= k <= n // 2
        assert G.shape == (k, (n + 63) // 64)
    ns = [n for _, n, _ in codes]
    assert min(ns) < 60 and max(ns) > 150
    again = I.batch_codes(count=5)
    assert all(np.array_equal(a[0], b[0]) for a, b in zip(again, codes[:5]))


def test_serving_trace_shapes():
    tr = I.serving_trace(400)
    times = [t for t, _, _, _ in tr]
    assert times == sorted(times)
    gaps = np.diff([0.0] + times)
    assert abs(gaps.mean() - 1 / 200.0) < 0.0015          # rate 200 / s
    for _, G, n, k in tr:
        assert 64 <= n <= 200 and abs(k - n // 2) <= 8
