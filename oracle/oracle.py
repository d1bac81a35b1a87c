"""ctypes front end of the C oracle (``md_oracle.c``).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module.  Nothing in the GPU library imports it, and it
imports nothing from the GPU library.

Matrices are numpy ``uint64`` arrays of shape (k, ceil(n/64)); bit t of word w of row i
is G[i, 64w + t].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OUT_D, OUT_KEY_G, OUT_KEY_J, OUT_KEY_RANK, OUT_L, OUT_M, OUT_STOP_G, OUT_STOP_J, \
    OUT_CODEWORDS, OUT_NLEVELS, OUT_COUNT = range(11)

ERRORS = {-1: "invalid argument", -2: "G is not of full row rank",
          -3: "level too large", -4: "out of memory"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile md_oracle.c into a shared library beside it (plain gcc, -O2), under a file
    lock so that concurrent processes build it once."""
    import fcntl
    os.makedirs(_BUILD, exist_ok=True)
    with open(os.path.join(_BUILD, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if (not force and os.path.exists(_LIB)
                    and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
                return _LIB
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
            return _LIB
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _bind(path: str):
    """Load a compiled oracle library and declare its entry points."""
    lib = ctypes.CDLL(path)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    i64p = ctypes.POINTER(ctypes.c_int64)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.mdo_binomial.restype = ctypes.c_uint64
    lib.mdo_binomial.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.mdo_colex_rank.restype = ctypes.c_uint64
    lib.mdo_colex_rank.argtypes = [ip, ctypes.c_int]
    lib.mdo_colex_next.restype = ctypes.c_int
    lib.mdo_colex_next.argtypes = [ip, ctypes.c_int, ctypes.c_int]
    lib.mdo_colex_unrank.restype = ctypes.c_int
    lib.mdo_colex_unrank.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ip]
    lib.mdo_rank.restype = ctypes.c_int
    lib.mdo_rank.argtypes = [u64p, ctypes.c_int, ctypes.c_int]
    lib.mdo_gamma.restype = ctypes.c_int
    lib.mdo_gamma.argtypes = [u64p, ctypes.c_int, ctypes.c_int, ip, u64p]
    lib.mdo_info_sets.restype = ctypes.c_int
    lib.mdo_info_sets.argtypes = [u64p, ctypes.c_int, ctypes.c_int, ip, ip]
    lib.mdo_bruteforce.restype = ctypes.c_int
    lib.mdo_bruteforce.argtypes = [u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]
    lib.mdo_scan.restype = ctypes.c_int
    lib.mdo_scan.argtypes = [u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                             ctypes.c_uint64, ctypes.c_int, ip, u64p]
    lib.mdo_bz.restype = ctypes.c_int
    lib.mdo_bz.argtypes = [u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           i64p, u64p, i64p, ctypes.c_int]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # MDO_ORACLE_LIB points at another build of md_oracle.c (the mutation tests
            # load deliberately broken copies this way)
            _lib = _bind(os.environ.get("MDO_ORACLE_LIB") or build())
        return _lib


def use_library(path: str):
    """Point this module at another compiled copy of md_oracle.c (returns the old one)."""
    global _lib
    with _lock:
        old = _lib
        _lib = _bind(path)
        return old


def restore_library(lib):
    global _lib
    with _lock:
        _lib = lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _check(rc):
    if rc < 0:
        raise OracleError(ERRORS.get(rc, "error %d" % rc))
    return rc


def words(n: int) -> int:
    return (n + 63) // 64


def binomial(a: int, b: int) -> int:
    return int(_load().mdo_binomial(a, b))


def colex_rank(c) -> int:
    arr = (ctypes.c_int * len(c))(*c)
    return int(_load().mdo_colex_rank(arr, len(c)))


def colex_next(c, k: int):
    """Colex successor of the sorted tuple c inside {0..k-1}, or None after the last."""
    arr = (ctypes.c_int * len(c))(*c)
    if not _load().mdo_colex_next(arr, len(c), k):
        return None
    return tuple(arr)


def colex_unrank(rank: int, g: int, k: int):
    arr = (ctypes.c_int * max(g, 1))()
    _check(_load().mdo_colex_unrank(rank, g, k, arr))
    return tuple(arr[:g])


def rank(G, n: int, k: int) -> int:
    G, p = _u64(G)
    return _check(_load().mdo_rank(p, n, k))


def info_sets(G, n: int, k: int):
    """(orders, ranks): per information set, the column order of its reduction and k_j."""
    G, p = _u64(G)
    orders = (ctypes.c_int * (n * n))()
    ranks = (ctypes.c_int * n)()
    m = _check(_load().mdo_info_sets(p, n, k, orders, ranks))
    return [list(orders[j * n:(j + 1) * n]) for j in range(m)], list(ranks[:m])


def gamma(G, n: int, k: int, order):
    """Reduced row echelon form of G with columns visited in `order`; (Gamma, pivots)."""
    G, p = _u64(G)
    out = np.zeros((k, words(n)), dtype=np.uint64)
    arr = (ctypes.c_int * n)(*order)
    piv = _check(_load().mdo_gamma(p, n, k, arr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return out, piv


def gammas(G, n: int, k: int):
    """All Gamma_j with their ranks k_j and column orders."""
    orders, ranks = info_sets(G, n, k)
    return [gamma(G, n, k, o)[0] for o in orders], ranks, orders


def bruteforce(G, n: int, k: int, threads: int = 1):
    """(d, dist): d = min weight over nonzero messages, dist[w] = #codewords of weight w."""
    G, p = _u64(G)
    dist = np.zeros(n + 1, dtype=np.uint64)
    d = _check(_load().mdo_bruteforce(p, n, k, threads,
                                      dist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
    return d, dist


def scan(Gam, n: int, k: int, g: int, r0: int, r1: int, threads: int = 1):
    """(min weight, first colex rank) over ranks [r0, r1) of level g of Gam."""
    Gam, p = _u64(Gam)
    w = ctypes.c_int()
    first = ctypes.c_uint64()
    _check(_load().mdo_scan(p, n, k, g, r0, r1, threads, ctypes.byref(w), ctypes.byref(first)))
    return w.value, first.value


class BZResult:
    def __init__(self, out, witness, levels):
        self.d = int(out[OUT_D])
        self.key = (int(out[OUT_KEY_G]), int(out[OUT_KEY_J]), int(out[OUT_KEY_RANK]))
        self.L = int(out[OUT_L])
        self.m = int(out[OUT_M])
        self.stop = (int(out[OUT_STOP_G]), int(out[OUT_STOP_J]))
        self.codewords = int(out[OUT_CODEWORDS])
        self.nlevels = int(out[OUT_NLEVELS])
        self.witness = witness
        # (g, j, min weight, first rank reaching it, combinations in the level)
        self.levels = [tuple(int(x) for x in row) for row in levels]

    def __repr__(self):
        return "BZResult(d=%d, key=%s, L=%d, m=%d, stop=%s, codewords=%d)" % (
            self.d, self.key, self.L, self.m, self.stop, self.codewords)


def bz(G, n: int, k: int, threads: int = 1, stop_after_g: int = 0, maxlev: int = 4096,
       stop_rule: int = 0) -> BZResult:
    """Plain Brouwer-Zimmermann (Alg. 1, bounds checked after each Gamma matrix);
    stop_rule 1 uses the per-matrix bound."""
    G, p = _u64(G)
    out = np.zeros(OUT_COUNT, dtype=np.int64)
    wit = np.zeros(words(n), dtype=np.uint64)
    lev = np.zeros((maxlev, 5), dtype=np.int64)
    i64 = ctypes.POINTER(ctypes.c_int64)
    _check(_load().mdo_bz(p, n, k, threads, stop_after_g, stop_rule, out.ctypes.data_as(i64),
                          wit.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                          lev.ctypes.data_as(i64), maxlev))
    nl = min(int(out[OUT_NLEVELS]), maxlev)
    return BZResult(out, wit, lev[:nl])
