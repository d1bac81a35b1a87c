"""Thin ctypes binding of the C ABI declared in include/md.h (same names, same meaning).

Only argument marshalling happens here: every step of the computation runs in
libmd.so.  The library is built in-tree by ``paper_1911_08963_gb300.build``; importing this
module without it raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MD_LIBRARY selects another build of the same library (the range-checked libmd_debug.so)
LIB_PATH = os.environ.get("MD_LIBRARY") or os.path.join(_HERE, "_lib", "libmd.so")

MD_OK, MD_EINVAL, MD_ERANK, MD_EUNSUPPORTED, MD_ENOMEM, MD_ECUDA, MD_EBUDGET, MD_ECANCELED, \
    MD_ETIMEOUT, MD_EBUSY, MD_EINTERNAL = range(11)
MD_MAX_N = 256
MD_MAX_GAMMA = 256
MD_MAX_LEVELS = 1024

# C prototypes, in the order of include/md.h.  Each entry: name -> (restype, argtypes).
u64p = ctypes.POINTER(ctypes.c_uint64)
ip = ctypes.POINTER(ctypes.c_int)


class md_options(ctypes.Structure):
    _fields_ = [("work_budget", ctypes.c_uint64), ("max_stage", ctypes.c_int), ("chunk_log2", ctypes.c_int),
                ("threads_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("filter", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("cancel_flag", ctypes.POINTER(ctypes.c_int)),
                ("batch_mode", ctypes.c_int), ("use_graph", ctypes.c_int), ("plan_horizon", ctypes.c_int),
                ("stop_rule", ctypes.c_int), ("perm_trials", ctypes.c_int), ("perm_seed", ctypes.c_uint64),
                ("tensor", ctypes.c_int), ("tensor_head", ctypes.c_int), ("test_stall", ctypes.c_int),
                ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p), ("alloc_ctx", ctypes.c_void_p),
                ("batch_heavy", ctypes.c_uint64), ("autotune", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("batch_workers", ctypes.c_int)]

# Prototypes of the allocator hook (md_options.dev_alloc / dev_free).
DEV_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEV_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class md_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("k", ctypes.c_int), ("m", ctypes.c_int),
                ("ranks", ctypes.c_int * MD_MAX_GAMMA), ("d", ctypes.c_int), ("complete", ctypes.c_int),
                ("lower_bound", ctypes.c_int), ("key_g", ctypes.c_int), ("key_j", ctypes.c_int),
                ("key_rank", ctypes.c_uint64), ("stop_g", ctypes.c_int), ("stop_j", ctypes.c_int),
                ("nlevels", ctypes.c_int), ("codewords", ctypes.c_uint64), ("seconds_total", ctypes.c_double),
                ("seconds_device", ctypes.c_double), ("gpu_launches", ctypes.c_int),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64), ("skipped_work", ctypes.c_uint64)]


class md_level(ctypes.Structure):
    _fields_ = [("g", ctypes.c_int), ("j", ctypes.c_int), ("weight", ctypes.c_int), ("words", ctypes.c_int),
                ("first_rank", ctypes.c_uint64), ("count", ctypes.c_uint64), ("seconds", ctypes.c_double)]


class md_task_info(ctypes.Structure):
    _fields_ = [("M", ctypes.c_uint32), ("per_lane", ctypes.c_uint32), ("uppers", ctypes.c_uint64),
                ("first_item", ctypes.c_uint64)]


class md_code(ctypes.Structure):
    _fields_ = [("G", u64p), ("n", ctypes.c_int), ("k", ctypes.c_int)]


class md_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("work_budget", ctypes.c_uint64), ("device_bytes", ctypes.c_size_t),
                ("stream", ctypes.c_void_p), ("stop_rule", ctypes.c_int), ("heavy", ctypes.c_uint64)]


PROTOTYPES = {
    "md_options_init": (ctypes.c_int, [ctypes.POINTER(md_options)]),
    "md_create": (ctypes.c_int, [u64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "md_create_ex": (ctypes.c_int, [u64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(md_options),
                                    ctypes.POINTER(ctypes.c_void_p)]),
    "md_compute": (ctypes.c_int, [ctypes.c_void_p, ip, u64p]),
    "md_checkpoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "md_resume": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "md_info_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(md_info)]),
    "md_levels": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(md_level), ctypes.c_int, ip]),
    "md_gamma": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, u64p, ip]),
    "md_scan_range": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                     ctypes.c_int, ip, u64p]),
    "md_scan_task": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_int, ip, u64p]),
    "md_level_plan": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ip, ctypes.POINTER(md_task_info),
                                     ctypes.c_int, ip, u64p]),
    "md_scan_range_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ip,
                                             u64p]),
    "md_popc_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "md_mma_rate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "md_debug_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
    "md_destroy": (None, [ctypes.c_void_p]),
    "md_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "md_batch": (ctypes.c_int, [ctypes.POINTER(md_code), ctypes.c_int, ctypes.POINTER(md_options), ip, u64p, ip]),
    "md_batch_tune": (ctypes.c_int, [ctypes.POINTER(md_code), ctypes.c_int, ctypes.POINTER(md_options),
                                     ctypes.c_char_p, ctypes.POINTER(md_options)]),
    "md_batch_tune_key": (ctypes.c_int, [ctypes.POINTER(md_code), ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]),
    "md_server_create": (ctypes.c_int, [ctypes.POINTER(md_server_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "md_server_submit": (ctypes.c_int, [ctypes.c_void_p, u64p, ctypes.c_int, ctypes.c_int, u64p]),
    "md_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ip, u64p, ip]),
    "md_server_destroy": (None, [ctypes.c_void_p]),
}

if not os.path.exists(LIB_PATH):
    raise ImportError("libmd.so is not built (%s); run `python -m paper_1911_08963_gb300.build` "
                      "or __graft_entry__.build()" % LIB_PATH)
lib = ctypes.CDLL(LIB_PATH)
for _name, (_res, _args) in PROTOTYPES.items():
    if hasattr(lib, _name):
        _f = getattr(lib, _name)
        _f.restype = _res
        _f.argtypes = _args


class MDError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, md_strerror(code), code))


def md_strerror(code: int) -> str:
    return lib.md_strerror(code).decode()


def _check(rc, where):
    if rc != MD_OK:
        if rc == MD_EINTERNAL and hasattr(lib, "md_debug_bounds"):
            debug, site = md_debug_bounds()
            if debug and site:
                where = "%s (range check failed at site %d)" % (where, site)
        raise MDError(rc, where)


def _rows(G, n, k):
    G = np.ascontiguousarray(G, dtype=np.uint64)
    if G.shape != (k, (n + 63) // 64):
        raise ValueError("G must have shape (k, ceil(n/64)) = (%d, %d), got %s" % (k, (n + 63) // 64, G.shape))
    return G, G.ctypes.data_as(u64p)


def md_options_init(**fields) -> md_options:
    o = md_options()
    _check(lib.md_options_init(ctypes.byref(o)), "md_options_init")
    for key, val in fields.items():
        setattr(o, key, val)
    return o


def md_create(G, n: int, k: int, options: md_options | None = None) -> int:
    G, p = _rows(G, n, k)
    h = ctypes.c_void_p()
    if options is None:
        _check(lib.md_create(p, n, k, ctypes.byref(h)), "md_create")
    else:
        _check(lib.md_create_ex(p, n, k, ctypes.byref(options), ctypes.byref(h)), "md_create_ex")
    return h.value


def md_compute(h: int, n: int):
    """(d, witness as uint64 words)."""
    d = ctypes.c_int()
    wit = np.zeros((n + 63) // 64, dtype=np.uint64)
    _check(lib.md_compute(h, ctypes.byref(d), wit.ctypes.data_as(u64p)), "md_compute")
    return d.value, wit


def md_checkpoint(h: int) -> bytes:
    """The state of the handle's last md_compute at its last completed level (include/md.h)."""
    size = ctypes.c_size_t()
    _check(lib.md_checkpoint(h, None, 0, ctypes.byref(size)), "md_checkpoint")
    buf = ctypes.create_string_buffer(max(1, size.value))
    _check(lib.md_checkpoint(h, buf, size.value, ctypes.byref(size)), "md_checkpoint")
    return buf.raw[:size.value]


def md_resume(h: int, ckpt: bytes) -> None:
    """Arm the handle's next md_compute to continue from a checkpoint."""
    buf = ctypes.create_string_buffer(ckpt, len(ckpt))
    _check(lib.md_resume(h, buf, len(ckpt)), "md_resume")


def md_info_get(h: int) -> dict:
    info = md_info()
    _check(lib.md_info_get(h, ctypes.byref(info)), "md_info_get")
    out = {f: getattr(info, f) for f, _ in md_info._fields_ if f != "ranks"}
    out["ranks"] = list(info.ranks[:info.m])
    return out


def md_levels(h: int, with_time: bool = False):
    """[(g, j, weight, first_rank, count)] (+ kernel seconds and product words if with_time)."""
    buf = (md_level * MD_MAX_LEVELS)()
    cnt = ctypes.c_int()
    _check(lib.md_levels(h, buf, MD_MAX_LEVELS, ctypes.byref(cnt)), "md_levels")
    if with_time:
        return [(r.g, r.j, r.weight, r.first_rank, r.count, r.seconds, r.words) for r in buf[:cnt.value]]
    return [(r.g, r.j, r.weight, r.first_rank, r.count) for r in buf[:cnt.value]]


def md_gamma(h: int, j: int, n: int, k: int):
    rows = np.zeros((k, (n + 63) // 64), dtype=np.uint64)
    order = (ctypes.c_int * n)()
    _check(lib.md_gamma(h, j, rows.ctypes.data_as(u64p), order), "md_gamma")
    return rows, list(order)


def md_scan_range(h: int, g: int, j: int, r0: int, r1: int, bound: int = -1):
    w = ctypes.c_int()
    r = ctypes.c_uint64()
    _check(lib.md_scan_range(h, g, j, r0, r1, bound, ctypes.byref(w), ctypes.byref(r)), "md_scan_range")
    return w.value, r.value


def md_scan_task(h: int, g: int, j: int, M: int, u0: int, u1: int, bound: int = -1):
    w = ctypes.c_int()
    r = ctypes.c_uint64()
    _check(lib.md_scan_task(h, g, j, M, u0, u1, bound, ctypes.byref(w), ctypes.byref(r)), "md_scan_task")
    return w.value, r.value


def md_level_plan(h: int, g: int, j: int):
    """(kind, [(M, per_lane, uppers, first_item)], work_items)."""
    kind = ctypes.c_int()
    cnt = ctypes.c_int()
    items = ctypes.c_uint64()
    buf = (md_task_info * 512)()
    _check(lib.md_level_plan(h, g, j, ctypes.byref(kind), buf, 512, ctypes.byref(cnt), ctypes.byref(items)),
           "md_level_plan")
    return kind.value, [(t.M, t.per_lane, t.uppers, t.first_item) for t in buf[:cnt.value]], items.value


def md_scan_range_noalloc(rows_ptr: int, k: int, words: int, weight_base: int, g: int, r0: int, r1: int,
                          bound: int = -1, stream=None):
    """rows_ptr: device address of the packed rows (see include/md.h)."""
    w = ctypes.c_int()
    r = ctypes.c_uint64()
    _check(lib.md_scan_range_noalloc(rows_ptr, k, words, weight_base, g, r0, r1, bound, stream, ctypes.byref(w),
                                     ctypes.byref(r)), "md_scan_range_noalloc")
    return w.value, r.value


def md_popc_rate() -> float:
    """POPC lane-operations per SM per clock on the current GPU (include/md.h)."""
    r = ctypes.c_double()
    _check(lib.md_popc_rate(ctypes.byref(r)), "md_popc_rate")
    return r.value


def md_mma_rate() -> float:
    """Dense e4m3 tensor-pipe flops per SM per clock on the current GPU (include/md.h)."""
    r = ctypes.c_double()
    _check(lib.md_mma_rate(ctypes.byref(r)), "md_mma_rate")
    return r.value


def md_debug_bounds():
    """(is the range-checked build, last failing check site or 0)."""
    site = ctypes.c_uint()
    rc = lib.md_debug_bounds(ctypes.byref(site))
    return rc == MD_OK, site.value


def md_destroy(h: int) -> None:
    if h:
        lib.md_destroy(h)


def _code_array(codes):
    """ctypes md_code array of [(G, n, k)] and the numpy rows it points into (keep alive)."""
    arr = (md_code * len(codes))()
    keep = []
    for i, (G, n, k) in enumerate(codes):
        G, p = _rows(G, n, k)
        keep.append(G)
        arr[i].G, arr[i].n, arr[i].k = p, n, k
    return arr, keep


def md_batch_tune(codes, options: md_options | None = None, cache_path: str | None = None) -> md_options:
    """The tuned copy of `options` (see include/md.h)."""
    arr, keep = _code_array(codes)
    out = md_options()
    _check(lib.md_batch_tune(arr, len(codes), ctypes.byref(options) if options is not None else None,
                             cache_path.encode() if cache_path else None, ctypes.byref(out)), "md_batch_tune")
    return out


def md_batch_tune_key(codes) -> str:
    arr, keep = _code_array(codes)
    buf = ctypes.create_string_buffer(256)
    _check(lib.md_batch_tune_key(arr, len(codes), buf, 256), "md_batch_tune_key")
    return buf.value.decode()


def md_batch(codes, options: md_options | None = None):
    """codes: list of (G, n, k).  Returns (d list, witnesses list, status list)."""
    arr, keep = _code_array(codes)
    offs = []
    total = 0
    for G, n, k in codes:
        offs.append(total)
        total += (n + 63) // 64
    d = (ctypes.c_int * len(codes))()
    st = (ctypes.c_int * len(codes))()
    wit = np.zeros(max(1, total), dtype=np.uint64)
    opt = ctypes.byref(options) if options is not None else None
    _check(lib.md_batch(arr, len(codes), opt, d, wit.ctypes.data_as(u64p), st), "md_batch")
    wits = [wit[o:o + (n + 63) // 64].copy() for o, (_, n, _) in zip(offs, codes)]
    return list(d), wits, list(st)


def md_server_create(slots: int = 0, work_budget: int = 0, device_bytes: int = 0, stream=None,
                     stop_rule: int = 0, heavy: int = 0) -> int:
    o = md_server_opts(slots, work_budget, device_bytes, stream, stop_rule, heavy)
    s = ctypes.c_void_p()
    _check(lib.md_server_create(ctypes.byref(o), ctypes.byref(s)), "md_server_create")
    return s.value


def md_server_submit(s: int, G, n: int, k: int) -> int:
    G, p = _rows(G, n, k)
    t = ctypes.c_uint64()
    _check(lib.md_server_submit(s, p, n, k, ctypes.byref(t)), "md_server_submit")
    return t.value


def md_server_poll(s: int, ticket: int, n: int):
    """None while pending, else (d, witness, status)."""
    d = ctypes.c_int()
    st = ctypes.c_int()
    wit = np.zeros((n + 63) // 64, dtype=np.uint64)
    rc = lib.md_server_poll(s, ticket, ctypes.byref(d), wit.ctypes.data_as(u64p), ctypes.byref(st))
    if rc == MD_EBUSY:
        return None
    _check(rc, "md_server_poll")
    return d.value, wit, st.value


def md_server_destroy(s: int) -> None:
    if s:
        lib.md_server_destroy(s)


def minimum_distance(G, n: int, k: int, **options):
    """Convenience wrapper: (d, witness, info, levels) for one code."""
    opt = md_options_init(**options) if options else None
    h = md_create(G, n, k, opt)
    try:
        d, wit = md_compute(h, n)
        return d, wit, md_info_get(h), md_levels(h)
    finally:
        md_destroy(h)
