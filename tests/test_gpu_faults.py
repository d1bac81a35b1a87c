"""GPU: failure paths injected on the host -- nothing here faults, traps or hangs a GPU.

  * Cancellation: another thread sets md_options.cancel_flag while md_compute runs; the
    calling thread passes it on to the kernels (a mapped pinned word checked before every work
    item), so the call returns MD_ECANCELED within a bounded time, long before the run would
    end, and the same handle then gives the exact result.
  * Allocation failure: the caller's device allocator (md_options.dev_alloc) returns NULL, so
    md_compute and md_batch return MD_ENOMEM; a working caller allocator (torch's) serves every
    device buffer, and the results are exact.
  * Checkpoint and resume: a run cancelled mid-level, or stopped at a stage limit, is
    checkpointed at its last completed level, resumed in another handle, and gives exactly the
    uninterrupted run's d, witness and level records.
"""
import ctypes
import os
import threading
import time

import numpy as np
import pytest

import oracle as O
from paper_1911_08963_gb300 import inputs as I

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def B():
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding
    return binding


def levels_of(B, G, n, k, **opts):
    h = B.md_create(G, n, k, B.md_options_init(**opts))
    try:
        d, wit = B.md_compute(h, n)
        return d, wit, B.md_levels(h)
    finally:
        B.md_destroy(h)


@pytest.mark.parametrize("tensor,delay", [(1, 1.0), (0, 0.5)])
def test_cancel_mid_run(B, tensor, delay):
    """[200,100] up to stage 10 takes ~3 s on the tensor cores (~10 s on the popcount kernels);
    the flag is set `delay` seconds in, inside the stage-10 (or stage-9) levels."""
    G, n, k = I.single_code("rand200x100")
    flag = ctypes.c_int(0)
    opt = B.md_options_init(max_stage=10, tensor=tensor)
    opt.cancel_flag = ctypes.pointer(flag)
    h = B.md_create(G, n, k, opt)
    try:
        timer = threading.Timer(delay, lambda: setattr(flag, "value", 1))
        t0 = time.perf_counter()
        timer.start()
        with pytest.raises(B.MDError) as e:
            B.md_compute(h, n)
        elapsed = time.perf_counter() - t0
        timer.join()
        assert e.value.code == B.MD_ECANCELED
        assert elapsed < delay + 0.5, elapsed             # stopped within ~one work item per warp
        # the same handle, flag cleared: the complete run, equal to a fresh handle's
        flag.value = 0
        d, wit = B.md_compute(h, n)
        lev = B.md_levels(h)
    finally:
        B.md_destroy(h)
    d2, wit2, lev2 = levels_of(B, G, n, k, max_stage=10, tensor=tensor)
    assert (d, lev) == (d2, lev2) and np.array_equal(wit, wit2)
    # and the first stages equal the oracle's records
    res = O.bz(G, n, k, threads=THREADS, stop_after_g=5)
    U = n + 1
    for got, (g, j, w, first, count) in zip(lev, res.levels):
        assert tuple(got) == ((g, j, w, first, count) if w <= U else (g, j, -1, 0, count))
        U = min(U, w)


def test_cancel_before_run(B):
    G, n, k = I.single_code("rand64x32")
    flag = ctypes.c_int(1)
    opt = B.md_options_init()
    opt.cancel_flag = ctypes.pointer(flag)
    h = B.md_create(G, n, k, opt)
    try:
        with pytest.raises(B.MDError) as e:
            B.md_compute(h, n)
        assert e.value.code == B.MD_ECANCELED
    finally:
        B.md_destroy(h)


class TorchAllocator:
    """A caller-owned device allocator: every buffer the library asks for is a torch tensor."""

    def __init__(self, fail=False):
        import torch
        self.torch = torch
        self.fail = fail
        self.live = {}
        self.calls = 0
        self.alloc_fn = None
        self.free_fn = None

    def options(self, B, **fields):
        def alloc(nbytes, ctx):
            self.calls += 1
            if self.fail:
                return None
            t = self.torch.empty(max(int(nbytes), 1), dtype=self.torch.uint8, device="cuda")
            self.live[t.data_ptr()] = t
            return t.data_ptr()

        def free(ptr, ctx):
            self.live.pop(ptr, None)

        self.alloc_fn = B.DEV_ALLOC(alloc)           # kept alive as long as the allocator
        self.free_fn = B.DEV_FREE(free)
        opt = B.md_options_init(**fields)
        opt.dev_alloc = ctypes.cast(self.alloc_fn, ctypes.c_void_p)
        opt.dev_free = ctypes.cast(self.free_fn, ctypes.c_void_p)
        return opt


def test_allocator_failure_is_enomem(B):
    pytest.importorskip("torch")
    G, n, k = I.single_code("rand64x32")
    A = TorchAllocator(fail=True)
    h = B.md_create(G, n, k, A.options(B))
    try:
        with pytest.raises(B.MDError) as e:
            B.md_compute(h, n)
        assert e.value.code == B.MD_ENOMEM
    finally:
        B.md_destroy(h)
    assert A.calls >= 1
    with pytest.raises(B.MDError) as e:
        B.md_batch(I.batch_codes(count=8), A.options(B))
    assert e.value.code == B.MD_ENOMEM


def test_caller_allocator_serves_every_buffer(B):
    pytest.importorskip("torch")
    G, n, k = I.single_code("rand64x32")
    res = O.bz(G, n, k)
    A = TorchAllocator()
    h = B.md_create(G, n, k, A.options(B, tensor=2, tensor_head=3))
    try:
        d, wit = B.md_compute(h, n)
        assert A.calls >= 1 and A.live
    finally:
        B.md_destroy(h)
    assert not A.live                                  # md_destroy returned every buffer
    assert d == res.d and np.array_equal(wit, res.witness)
    codes = [c for c in I.batch_codes(count=64) if c[1] <= 100][:12]      # within the oracle's reach
    d_b, w_b, st_b = B.md_batch(codes, A.options(B))
    assert not A.live
    for (Gc, nc, kc), dc, wc, sc in zip(codes, d_b, w_b, st_b):
        assert sc == B.MD_OK
        r = O.bz(Gc, nc, kc, threads=THREADS)
        assert dc == r.d and np.array_equal(wc, r.witness)


def test_resume_after_cancel_equals_uninterrupted(B):
    """Cancel [200,100] (stages <= 10, tensor cores) one second in, checkpoint, resume in a new
    handle: the same d, witness and every level record as an uninterrupted run; the checkpoint
    holds only levels the cancelled run completed."""
    G, n, k = I.single_code("rand200x100")
    flag = ctypes.c_int(0)
    opt = B.md_options_init(max_stage=10)
    opt.cancel_flag = ctypes.pointer(flag)
    h = B.md_create(G, n, k, opt)
    try:
        timer = threading.Timer(1.0, lambda: setattr(flag, "value", 1))
        timer.start()
        with pytest.raises(B.MDError) as e:
            B.md_compute(h, n)
        timer.join()
        assert e.value.code == B.MD_ECANCELED
        ckpt = B.md_checkpoint(h)
    finally:
        B.md_destroy(h)
    nlev = (len(ckpt) - 48) // 12
    assert 0 < nlev < 20                          # stopped inside stage 10 (levels 18, 19)
    d2, wit2, lev2 = levels_of(B, G, n, k, max_stage=10)
    h = B.md_create(G, n, k, B.md_options_init(max_stage=10))
    try:
        B.md_resume(h, ckpt)
        d, wit = B.md_compute(h, n)
        lev = B.md_levels(h)
        info = B.md_info_get(h)
    finally:
        B.md_destroy(h)
    assert d == d2 and np.array_equal(wit, wit2) and lev == lev2
    assert info["codewords"] == sum(x[4] for x in lev2)


def test_resume_extends_a_stage_limited_run(B):
    """A run stopped at max_stage = 6, resumed with max_stage = 8, equals a max_stage = 8 run;
    the first stages equal the oracle's records, and a checkpoint of another code is refused."""
    G, n, k = I.single_code("rand200x100")
    h = B.md_create(G, n, k, B.md_options_init(max_stage=6))
    try:
        B.md_compute(h, n)
        ckpt = B.md_checkpoint(h)
    finally:
        B.md_destroy(h)
    h = B.md_create(G, n, k, B.md_options_init(max_stage=8))
    try:
        B.md_resume(h, ckpt)
        d, wit = B.md_compute(h, n)
        lev = B.md_levels(h)
    finally:
        B.md_destroy(h)
    d2, wit2, lev2 = levels_of(B, G, n, k, max_stage=8)
    assert d == d2 and np.array_equal(wit, wit2) and lev == lev2
    res = O.bz(G, n, k, threads=THREADS, stop_after_g=5)
    U = n + 1
    for got, (g, j, w, first, count) in zip(lev, res.levels):
        assert tuple(got) == ((g, j, w, first, count) if w <= U else (g, j, -1, 0, count))
        U = min(U, w)
    G2, n2, k2 = I.single_code("rand128x64")
    h = B.md_create(G2, n2, k2)
    try:
        with pytest.raises(B.MDError) as e:
            B.md_resume(h, ckpt)
        assert e.value.code == B.MD_EINVAL
    finally:
        B.md_destroy(h)
