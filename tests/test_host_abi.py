"""CPU-side checks of the C ABI library: it loads, exports every entry point declared in
include/md.h, validates its inputs, and builds the same Gamma_j as the oracle, bit for bit.
No call here touches the GPU (md_create and md_gamma are host-only)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from tests import textbook as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_1911_08963_gb300 import build
    build.build()
    from paper_1911_08963_gb300 import binding
    return binding


def declared_functions():
    src = open(os.path.join(ROOT, "include", "md.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(md_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(B):
    names = declared_functions()
    assert "md_compute" in names and "md_batch" in names and "md_server_poll" in names
    missing = [n for n in names if not hasattr(B.lib, n)]
    assert not missing, missing
    assert set(names) <= set(B.PROTOTYPES)


def test_strerror(B):
    for code in range(11):
        assert B.md_strerror(code)
    assert B.md_strerror(999) == "unknown status"


def test_create_validation(B):
    rows = T.random_rows(40, 10, 1)
    G = T.pack(rows, 40)
    h = B.md_create(G, 40, 10)
    B.md_destroy(h)
    with pytest.raises(B.MDError) as e:
        B.md_create(T.pack(rows[:9] + [rows[0] ^ rows[1]], 40), 40, 10)
    assert e.value.code == B.MD_ERANK
    # any padding bit set: the first one (column n), one further on, the last of the word,
    # and a padding bit in the last word of a wider row (n = 130: columns 130..191)
    for n_, k_, word, bit in ((40, 10, 0, 40), (40, 10, 0, 45), (40, 10, 0, 63), (130, 20, 2, 2), (130, 20, 2, 63)):
        rows_ = T.random_rows(n_, k_, 2)
        bad = T.pack(rows_, n_)
        B.md_destroy(B.md_create(bad, n_, k_))               # valid without the bit
        bad[k_ - 1, word] |= np.uint64(1 << bit)
        with pytest.raises(B.MDError) as e:
            B.md_create(bad, n_, k_)
        assert e.value.code == B.MD_EINVAL, (n_, word, bit)
    big = np.zeros((1, 5), dtype=np.uint64)
    big[0, 0] = 1
    with pytest.raises(B.MDError) as e:
        B.md_create(big, 257, 1)
    assert e.value.code == B.MD_EUNSUPPORTED
    p = G.ctypes.data_as(B.u64p)
    hh = ctypes.c_void_p()
    assert B.lib.md_create(p, 40, 41, ctypes.byref(hh)) == B.MD_EINVAL
    assert B.lib.md_create(p, 0, 0, ctypes.byref(hh)) == B.MD_EINVAL
    assert B.lib.md_create(None, 40, 10, ctypes.byref(hh)) == B.MD_EINVAL


@pytest.mark.parametrize("n,k,seed", [(16, 5, 1), (24, 8, 2), (40, 13, 3), (70, 20, 4), (130, 40, 5),
                                      (64, 32, 6), (9, 9, 7), (33, 1, 8), (200, 100, 9), (256, 100, 10),
                                      (256, 150, 11), (250, 7, 12), (97, 48, 13), (160, 80, 14)])
def test_gamma_bit_exact_with_oracle(B, n, k, seed):
    rows = T.random_rows(n, k, seed)
    G = T.pack(rows, n)
    gams, ranks, orders = O.gammas(G, n, k)
    h = B.md_create(G, n, k)
    try:
        info = B.md_info_get(h)
        assert info["m"] == len(gams) and info["ranks"] == ranks
        for j in range(len(gams)):
            rows_j, order_j = B.md_gamma(h, j, n, k)
            assert order_j == orders[j]
            assert np.array_equal(rows_j, gams[j]), (n, k, j)
    finally:
        B.md_destroy(h)


def test_gamma_leftover_sets_match_oracle(B):
    """The library's information sets follow the oracle on codes built to have a leftover set
    of rank 1 ([I_4 | I_4 | e_0]: three matrices, ranks 4, 4, 1) and an all-zero leftover
    column ([I_4 | I_4 | 0]: two matrices): the same m, ranks, column orders and Gamma_j."""
    k, n = 4, 9
    for last, want in ((1, [4, 4, 1]), (0, [4, 4])):
        rows = [(1 << i) | (1 << (k + i)) | ((last << (2 * k)) if i == 0 else 0) for i in range(k)]
        G = T.pack(rows, n)
        gams, ranks, orders = O.gammas(G, n, k)
        assert ranks == want
        h = B.md_create(G, n, k)
        try:
            info = B.md_info_get(h)
            assert info["m"] == len(want) and info["ranks"] == want
            for j in range(len(want)):
                rj, oj = B.md_gamma(h, j, n, k)
                assert np.array_equal(rj, gams[j]) and oj == orders[j], (last, j)
        finally:
            B.md_destroy(h)


def test_gamma_textbook(B):
    for name, (ctor, d, _) in T.TEXTBOOK.items():
        rows, n, k = ctor()
        G = T.pack(rows, n)
        gams, ranks, orders = O.gammas(G, n, k)
        h = B.md_create(G, n, k)
        try:
            for j in range(len(gams)):
                rj, oj = B.md_gamma(h, j, n, k)
                assert np.array_equal(rj, gams[j]) and oj == orders[j], name
        finally:
            B.md_destroy(h)


@pytest.mark.parametrize("n,k,g", [(100, 33, 6), (200, 100, 10), (200, 100, 5), (160, 80, 8), (64, 32, 4),
                                   (256, 150, 6), (48, 24, 7), (128, 64, 7)])
def test_level_plan_covers_every_combination(B, n, k, g):
    """The split decomposition covers C(k, g) combinations: sum over M of
    C(k-1-M, v) upper parts times C(M, P) heads (closed form), work items are contiguous,
    and every work item holds at most 32 lanes x per_lane upper parts.  (tensor = 0: the
    popcount kernels' plan, which large levels use without the tensor cores.)"""
    import math
    rows = T.random_rows(n, k, 3)
    h = B.md_create(T.pack(rows, n), n, k, B.md_options_init(tensor=0))
    try:
        kind, tasks, items = B.md_level_plan(h, g, 0)
        if g <= 4:
            assert kind == 0 and tasks == [] and items >= 1
            return
        P = kind
        assert P == (2 if g == 5 else 3)
        v = g - P - 1
        total = 0
        next_item = 0
        assert [t[0] for t in tasks] == list(range(P, k - v))
        for M, per_lane, uppers, first in tasks:
            assert uppers == math.comb(k - 1 - M, v)
            assert first == next_item
            next_item += -(-uppers // (32 * per_lane))
            total += uppers * math.comb(M, P)
        assert next_item == items
        assert total == math.comb(k, g)
    finally:
        B.md_destroy(h)


def _tc_items(k, g, q, W):
    """Work items of a tensor-core level and the combinations they cover, restated from the
    two-phase split: phase 0 takes c_{q+1} = s >= s_min with the C(s, q) q-heads below s,
    phase 1 takes c_{q+1} < s_min with (q+1)-heads below min(c_{q+2}, s_min); each s is
    cut into groups of up to 16 slices of 256 heads times runs of up to 128 T tails."""
    import math
    T_ = 8 if W <= 2 else 4 if W <= 4 else 2 if W <= 6 else 1
    smin = q
    if g >= q + 2:
        while smin < k and math.comb(smin, q) < 7 * 256:
            smin += 1
    items = cover = 0
    for ph in (0, 1):
        qq, v = q + ph, g - q - ph - 1
        if v < 0:
            continue
        for s in range(qq if ph else max(q, smin), k - v):
            nb = math.comb(min(s, smin), qq) if ph else math.comb(s, qq)
            nt = math.comb(k - 1 - s, v)
            items += -(-(-(-nb // 256)) // 16) * -(-nt // (128 * T_))
            cover += nb * nt
    return items, cover


def _auto_q(k, W):
    """The automatic head size: the widest of 5, 4, 3 elements whose table (C(k, q) heads
    in 256-row slices of 32 W bytes) fits in 1 GiB, else 2."""
    import math
    for q in (5, 4, 3):
        if k > q + 1 and -(-math.comb(k, q) // 256) * 256 * 32 * W <= 1 << 30:
            return q
    return 2


@pytest.mark.parametrize("n,k,g,head,tensor", [(200, 100, 8, 0, 1), (200, 100, 10, 0, 1), (128, 64, 7, 0, 1),
                                               (256, 60, 6, 0, 2), (100, 33, 4, 3, 2), (120, 40, 6, 2, 2),
                                               (90, 30, 9, 0, 2), (160, 60, 12, 0, 1), (200, 100, 9, 3, 1),
                                               (150, 60, 13, 4, 1), (120, 50, 9, 5, 2)])
def test_level_plan_tensor_items(B, n, k, g, head, tensor):
    """Levels md_compute runs on the tensor cores report kind 4; the item count matches the
    two-phase split restated here, and the two phases cover the C(k, g) combinations once."""
    import math
    h = B.md_create(T.pack(T.random_rows(n, k, 5), n), n, k, B.md_options_init(tensor=tensor, tensor_head=head))
    try:
        kind, tasks, items = B.md_level_plan(h, g, 0)
    finally:
        B.md_destroy(h)
    W = -(-(n - k) // 32)
    q = head or _auto_q(k, W)
    want, cover = _tc_items(k, g, q, W)
    assert kind == 4 and tasks == []
    assert items == want
    assert cover == math.comb(k, g)


def test_level_plan_small_enumeration_exact(B):
    """Tiny level: the combinations generated from the plan (heads below M, M, upper part
    by colex index) are exactly the g-subsets, each with its colex rank."""
    import math
    import itertools
    n, k, g = 50, 28, 6                  # C(28, 6) = 376740 >= 2^18: a split level
    h = B.md_create(T.pack(T.random_rows(n, k, 4), n), n, k)
    try:
        kind, tasks, items = B.md_level_plan(h, g, 0)
    finally:
        B.md_destroy(h)
    assert kind == 3
    P = 3
    v = g - P - 1
    got = []
    for M, per_lane, uppers, first in tasks:
        for u in range(uppers):
            up = tuple(M + 1 + e for e in O.colex_unrank(u, v, k - 1 - M))
            for head in itertools.combinations(range(M), P):
                c = head + (M,) + up
                got.append((T.colex_rank_formula(c), c))
    assert sorted(r for r, _ in got) == list(range(math.comb(k, g)))
    assert sorted(c for _, c in got) == list(itertools.combinations(range(k), g))


def test_struct_layouts_match_header(B, tmp_path):
    """The binding's ctypes mirrors have the sizes and field offsets of include/md.h (gcc
    compiles a probe that prints them).  A drift would let the library write past a struct
    that Python owns, as md_options_init does with the whole of md_options."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    structs = [B.md_options, B.md_info, B.md_level, B.md_task_info, B.md_code, B.md_server_opts]
    lines = ["#include <stdio.h>", "#include \"md.h\"", "int main(void) {"]
    for S in structs:
        name = S.__name__
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in S._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for S in structs:
        assert int(got["%s size" % S.__name__]) == ctypes.sizeof(S), S.__name__
        for f, _ in S._fields_:
            assert int(got["%s.%s" % (S.__name__, f)]) == getattr(S, f).offset, (S.__name__, f)


@pytest.mark.parametrize("n,k,g,tensor,why", [(200, 60, 17, 2, "v = 11 upper elements (q = 5)"),
                                              (200, 100, 5, 1, "C(100, 5) < 2^28"),
                                              (200, 100, 10, 0, "tensor = 0")])
def test_level_plan_tensor_fallbacks(B, n, k, g, tensor, why):
    """Levels the tensor-core kernel does not take keep the split plan: tails of more than
    10 upper elements (g - q - 1 > 10), levels below 2^28 combinations under the default
    rule, and tensor = 0."""
    h = B.md_create(T.pack(T.random_rows(n, k, 6), n), n, k, B.md_options_init(tensor=tensor))
    try:
        kind, tasks, items = B.md_level_plan(h, g, 0)
    finally:
        B.md_destroy(h)
    assert kind in (2, 3), why
    assert tasks and items >= 1


@pytest.mark.parametrize("k,g,q,smin", [(12, 6, 3, 6), (13, 7, 2, 5), (11, 5, 3, 4), (10, 4, 3, 3), (12, 9, 3, 7)])
def test_tensor_split_heads_are_colex_prefixes(k, g, q, smin):
    """Brute force over all g-subsets, ranks from the oracle's colex rank: the heads the
    tensor-core kernel pairs with a tail are a colex prefix of the head table (phase 0: the
    q-subsets below s = c_{q+1} are the first C(s, q); phase 1: the (q+1)-subsets below
    min(c_{q+2}, s_min) are the first C(min(c_{q+2}, s_min), q+1)), the rank splits into head
    index + tail part, and the two phases meet every combination once."""
    import itertools
    import math
    heads = {r: sorted(itertools.combinations(range(k), r), key=O.colex_rank) for r in (q, q + 1)}
    seen = set()
    for c in itertools.combinations(range(k), g):
        if c[q] >= smin:                                   # phase 0: tail c_{q+1}..c_g
            s, head, r = c[q], c[:q], q
            allowed = math.comb(s, q)
        else:                                              # phase 1: tail c_{q+2}..c_g
            if g < q + 2:
                continue
            s, head, r = c[q + 1], c[:q + 1], q + 1
            allowed = math.comb(min(s, smin), q + 1)
        p = heads[r].index(head)
        assert p < allowed
        assert all(max(h) < min(s, smin) if r == q + 1 else max(h) < s for h in heads[r][:allowed])
        tail = O.colex_rank(c) - O.colex_rank(head)
        assert O.colex_rank(c) == p + tail
        seen.add(c)
    assert len(seen) == math.comb(k, g)                   # (s_min = q when g < q + 2, as planned)


def test_batch_tune_key_and_no_gpu(B):
    """The tuning key names the batch's shape (n and k rounded out, count to a power of two);
    without a GPU the tuner reports MD_ECUDA rather than guessing."""
    codes = [(T.pack(T.random_rows(n, k, 40 + i), n), n, k) for i, (n, k) in enumerate([(50, 20), (97, 41), (130, 60)])]
    assert B.md_batch_tune_key(codes) == "n48-144 k16-64 c2^2"
    assert B.md_batch_tune_key(codes[:1]) == "n48-64 k16-24 c2^0"
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(B.MDError) as e:
            B.md_batch_tune(codes)
        assert e.value.code == B.MD_ECUDA


def test_checkpoint_and_resume_reject_what_they_cannot_use(B):
    """md_checkpoint needs a finished md_compute on the handle; md_resume checks its buffer
    (size, magic, the code and stop rule it was taken from) and takes nothing else."""
    n, k = 40, 12
    h = B.md_create(T.pack(T.random_rows(n, k, 3), n), n, k)
    try:
        with pytest.raises(B.MDError) as e:
            B.md_checkpoint(h)
        assert e.value.code == B.MD_EINVAL
        for junk in (b"", b"x" * 7, b"\0" * 48, b"MKCHPT01" + b"\0" * 40, b"\xff" * 200):
            with pytest.raises(B.MDError) as e:
                B.md_resume(h, junk)
            assert e.value.code == B.MD_EINVAL
    finally:
        B.md_destroy(h)
