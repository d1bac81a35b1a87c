"""GPU: distinct handles used at once from several host threads (the C ABI allows it) give
exactly the results of one-at-a-time runs, which the oracle confirms.

The codes pair equal packed row widths with different k, so that the same kernels are launched
from different threads with different shared-memory sizes: a kernel's shared-memory limit is
an attribute of the whole process, and a limit set per launch could be lowered by one thread
just before another thread's larger launch."""
import threading

import numpy as np
import pytest

import oracle as O
from tests import textbook as T

pytestmark = pytest.mark.gpu

# (n, k): n - k packed in 3 words for the first four, 2 words for the rest
SHAPES = [(126, 57), (100, 33), (110, 44), (90, 24), (80, 30), (70, 22), (64, 20), (60, 28)]


@pytest.fixture(scope="module")
def B():
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding
    return binding


def codes():
    return [(T.pack(T.random_rows(n, k, 700 + i), n), n, k) for i, (n, k) in enumerate(SHAPES)]


def run(B, G, n, k, opts):
    h = B.md_create(G, n, k, B.md_options_init(**opts))
    try:
        return B.md_compute(h, n)
    finally:
        B.md_destroy(h)


@pytest.mark.parametrize("opts", [{"tensor": 2, "tensor_head": 3}, {"tensor": 0}])
def test_handles_on_threads_equal_sequential_runs(B, opts):
    cs = codes()
    ref = [run(B, G, n, k, opts) for G, n, k in cs]
    for (G, n, k), (d, w) in zip(cs, ref):
        if k <= 30:
            res = O.bz(G, n, k, threads=8)
            assert d == res.d and np.array_equal(w, res.witness), (n, k)
    errors, results = [], {}

    def worker(t):
        try:
            for rep in range(3):
                for i in range(len(cs)):
                    j = (i + t) % len(cs)            # the threads start on different codes
                    G, n, k = cs[j]
                    results[(t, rep, j)] = run(B, G, n, k, opts)
        except Exception as e:                      # reported below, with the thread
            errors.append((t, repr(e)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for (t, rep, j), (d, w) in results.items():
        assert d == ref[j][0] and np.array_equal(w, ref[j][1]), (t, rep, SHAPES[j])
