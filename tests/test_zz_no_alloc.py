"""md_scan_range_noalloc: the rank-range scan for callers that cannot allocate device memory.

Such callers (real-time loops that forbid allocation after start-up, programs whose device
memory belongs to another allocator) pass their own device copy of the packed rows; the entry
point keeps its scratch in a fixed array inside the library.  This test checks, through the C
ABI, that consecutive calls give exactly what the CPU oracle's scan of the same colex ranks
gives, and what md_scan_range gives (the results are integers: tolerance zero).  It sits in a
file of its own that is collected last.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_08963_gb300 import inputs as I

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


def test_noalloc_scan_equals_oracle_and_scan_range_twice():
    torch = pytest.importorskip("torch")
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding as B

    G, n, k = I.single_code("rand200x100")
    h = B.md_create(G, n, k)
    try:
        gam, _ = B.md_gamma(h, 1, n, k)
        # every column packed: 200 bits in 7 words, row stride 8 words (the uint64 rows as 32-bit words)
        rows32 = np.ascontiguousarray(gam).view(np.int32)
        assert rows32.shape == (k, 8)
        dev = torch.from_numpy(rows32.copy()).cuda()
        torch.cuda.synchronize()
        gams, _, _ = O.gammas(G, n, k)
        assert np.array_equal(gams[1], gam)
        cases = [(7, 10 ** 9, 10 ** 9 + 3 * 10 ** 6, -1), (4, 0, 3921225, -1),
                 (7, 10 ** 9, 10 ** 9 + 3 * 10 ** 6, 40), (7, 10 ** 9, 10 ** 9 + 3 * 10 ** 6, 60),
                 (3, 5, 5, -1)]
        for g, r0, r1, bound in cases:          # consecutive calls share the scratch array
            got = B.md_scan_range_noalloc(dev.data_ptr(), k, 7, 0, g, r0, r1, bound)
            want = B.md_scan_range(h, g, 1, r0, r1, bound)
            assert got == want, (g, r0, r1, bound, got, want)
            if r1 > r0:
                w, first = O.scan(gams[1], n, k, g, r0, r1, threads=THREADS)
                ref = (w, first) if bound < 0 or w <= bound else (-1, 0)
            else:
                ref = (-1, 0)
            assert got == ref, (g, r0, r1, bound, got, ref)
        with pytest.raises(B.MDError) as e:
            B.md_scan_range_noalloc(dev.data_ptr(), 129, 7, 0, 3, 0, 10)
        assert e.value.code == B.MD_EUNSUPPORTED
    finally:
        B.md_destroy(h)
