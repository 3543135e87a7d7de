"""Python binding of the C ABI in include/reach.h (ctypes; argument marshalling only).

Every computation runs in the CUDA library libvss.so; this module converts
arguments and raises on error codes.  It fails loudly when the library has not
been built: there is no CPU fallback.

Two layers:
  * functions named exactly like the C entry points (ht_create, ht_find_or_put,
    reach_ctx_run, reach, ...), taking raw pointers / ints;
  * `Table` and `ReachContext`, which take device memory from PyTorch tensors
    (torch is used for memory and streams only).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

(HT_OK, HT_ERR_INVALID, HT_ERR_OOM, HT_ERR_FULL, HT_ERR_TIMEOUT, HT_ERR_CUDA, HT_ERR_LEVELS,
 HT_ERR_TOO_BIG) = range(8)
REACH_PERSISTENT, REACH_PER_LEVEL, REACH_GRAPH, REACH_TRACE = 0, 1, 2, 4
STATUS_NAMES = {0: "HT_OK", 1: "HT_ERR_INVALID", 2: "HT_ERR_OOM", 3: "HT_ERR_FULL",
                4: "HT_ERR_TIMEOUT", 5: "HT_ERR_CUDA", 6: "HT_ERR_LEVELS", 7: "HT_ERR_TOO_BIG"}

EXPORTED = [
    "ht_bytes", "ht_create", "ht_create_at", "ht_destroy", "ht_clear", "ht_find_or_put", "ht_sync",
    "ht_stats", "ht_scan", "ht_gather", "ht_arrays", "ht_status_string",
    "reach_ctx_bytes", "reach_ctx_create", "reach_ctx_create_at", "reach_ctx_destroy",
    "reach_ctx_load", "reach_ctx_run", "reach_ctx_result", "reach_ctx_table", "reach",
    "reach_ctx_last_timing", "reach_ctx_level_ns", "vss_probe_random", "reach_noalloc",
    "vss_gen_keys", "ht_find_or_put_stream",
    "reach_batch_bytes", "reach_batch_create", "reach_batch_create_at", "reach_batch_destroy",
    "reach_batch_run", "reach_batch_results", "reach_batch_last_timing",
    "serve_bytes", "serve_open_at", "serve_open", "serve_submit", "serve_poll", "serve_status",
    "serve_close", "reach_ctx_deadlock_trace",
    "ht_bytes_n", "ht_create_n_at", "ht_buckets_for_bytes", "vss_line_divide",
    "reach_ctx_bytes_n", "reach_ctx_create_n_at", "reach_ctx_buckets_for_bytes",
    "reach_ctx_run_times", "vss_probe_random_cfg",
    "part_reach_bytes", "part_reach_create_at", "part_reach_destroy", "part_reach_run",
    "part_reach_last_exchange",
]


class HtError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {STATUS_NAMES.get(self.status, self.status)}")


class ht_params(ctypes.Structure):
    _fields_ = [("line_buckets", ctypes.c_uint32), ("max_rehash", ctypes.c_uint32),
                ("max_spin", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("dedup", ctypes.c_uint32), ("bucket_bits", ctypes.c_uint32),
                ("group_lanes", ctypes.c_uint32), ("rehash", ctypes.c_uint32),
                ("hash_seed", ctypes.c_uint64)]


class ht_stats_t(ctypes.Structure):
    _fields_ = [("stored", ctypes.c_uint64), ("busy_waits", ctypes.c_uint64),
                ("rehashes", ctypes.c_uint64), ("capacity", ctypes.c_uint64),
                ("error", ctypes.c_uint32), ("state_words", ctypes.c_uint32)]


_ip = ctypes.POINTER(ctypes.c_int32)


class reach_model(ctypes.Structure):
    _fields_ = [("n_procs", ctypes.c_int32), ("n_shared", ctypes.c_int32),
                ("state_words", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("n_local", _ip), ("crit", _ip), ("edge_begin", _ip), ("edge_dst", _ip),
                ("guard_var", _ip), ("guard_val", _ip), ("upd_var", _ip), ("upd_val", _ip)]


class reach_result(ctypes.Structure):
    _fields_ = [("states", ctypes.c_uint64), ("transitions", ctypes.c_uint64),
                ("deadlocks", ctypes.c_uint64), ("digest", ctypes.c_uint64),
                ("busy_waits", ctypes.c_uint64), ("rehashes", ctypes.c_uint64),
                ("n_levels", ctypes.c_uint32), ("status", ctypes.c_int32)]


_lib = None
_VP = ctypes.c_void_p
_u64 = ctypes.c_uint64
_i = ctypes.c_int
_st = ctypes.c_int32


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libvss.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    sig = {
        "ht_bytes": [_i, _i, ctypes.POINTER(_u64)],
        "ht_create": [_i, _i, ctypes.POINTER(ht_params), ctypes.POINTER(_VP)],
        "ht_create_at": [_i, _i, ctypes.POINTER(ht_params), _VP, _u64, ctypes.POINTER(_VP)],
        "ht_destroy": [_VP],
        "ht_clear": [_VP, _VP],
        "ht_find_or_put": [_VP, _VP, _u64, _VP, _VP, _VP],
        "ht_sync": [_VP, _VP],
        "ht_stats": [_VP, _VP, ctypes.POINTER(ht_stats_t)],
        "ht_scan": [_VP, _VP, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
        "ht_gather": [_VP, _VP, _u64, _VP, _VP],
        "ht_arrays": [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_uint32)],
        "reach_ctx_bytes": [_i, _i, ctypes.c_uint32, ctypes.POINTER(_u64)],
        "reach_ctx_create": [_i, _i, ctypes.c_uint32, ctypes.POINTER(ht_params), ctypes.POINTER(_VP)],
        "reach_ctx_create_at": [_i, _i, ctypes.c_uint32, ctypes.POINTER(ht_params), _VP, _u64,
                                ctypes.POINTER(_VP)],
        "reach_ctx_destroy": [_VP],
        "reach_ctx_load": [_VP, ctypes.POINTER(reach_model), _VP, _VP],
        "reach_ctx_run": [_VP, _i, _VP],
        "reach_ctx_result": [_VP, _VP, _VP, ctypes.c_uint32, ctypes.POINTER(reach_result)],
        "reach_ctx_table": [_VP, ctypes.POINTER(_VP)],
        "reach_ctx_last_timing": [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint32)],
        "reach_ctx_level_ns": [_VP, _VP, _VP, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)],
        "vss_probe_random": [_VP, _u64, _u64, _i, _VP, ctypes.POINTER(ctypes.c_float)],
        "vss_probe_random_cfg": [_VP, _u64, _u64, _i, _i, _i, _i, _VP, ctypes.POINTER(ctypes.c_float)],
        "part_reach_bytes": [_i, _i, _i, _u64, ctypes.POINTER(_u64)],
        "part_reach_create_at": [_i, _i, _i, _u64, ctypes.POINTER(ht_params), _VP, _u64,
                                 ctypes.POINTER(_VP)],
        "part_reach_destroy": [_VP],
        "part_reach_run": [_VP, ctypes.POINTER(reach_model), _VP, _VP, _VP, ctypes.c_uint32,
                           ctypes.POINTER(reach_result), _VP, ctypes.POINTER(_u64)],
        "part_reach_last_exchange": [_VP, _VP, _VP, _VP],
        "vss_gen_keys": [_u64, _u64, _u64, _u64, _VP, _i, _VP, _VP],
        "ht_find_or_put_stream": [_VP, _u64, _u64, _u64, _u64, _VP, _VP, _VP],
        "reach_batch_bytes": [_VP, _VP, _i, ctypes.c_uint32, _u64, ctypes.POINTER(_u64)],
        "reach_batch_create_at": [_VP, _VP, _i, _VP, ctypes.c_uint32, _u64, ctypes.POINTER(ht_params),
                                  _VP, _u64, ctypes.POINTER(_VP)],
        "reach_batch_create": [_VP, _VP, _i, _VP, ctypes.c_uint32, _u64, ctypes.POINTER(ht_params),
                               ctypes.POINTER(_VP)],
        "reach_batch_destroy": [_VP],
        "reach_batch_run": [_VP, _i, _VP],
        "reach_batch_results": [_VP, _VP, _VP, _VP, _VP],
        "reach_batch_last_timing": [_VP, ctypes.POINTER(ctypes.c_float)],
        "serve_bytes": [_u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(_u64)],
        "serve_open_at": [_VP, _u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ht_params),
                          ctypes.POINTER(_VP)],
        "serve_open": [_u64, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ht_params),
                       ctypes.POINTER(_VP)],
        "serve_submit": [_VP, ctypes.POINTER(reach_model), _VP, _i, ctypes.POINTER(_u64)],
        "serve_poll": [_VP, _VP, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32), _VP],
        "serve_status": [_VP, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                         ctypes.POINTER(_u64), ctypes.POINTER(_u64)],
        "serve_close": [_VP],
        "reach_ctx_deadlock_trace": [_VP, _VP, _VP, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                                     ctypes.POINTER(ctypes.c_uint32)],
        "reach_noalloc": [ctypes.POINTER(reach_model), _VP, _i, ctypes.POINTER(ht_params), _VP, _VP,
                          ctypes.c_uint32, ctypes.POINTER(reach_result)],
        "reach": [_VP, ctypes.POINTER(reach_model), _VP, _i, _VP, _VP, ctypes.c_uint32,
                  ctypes.POINTER(reach_result)],
        "reach_ctx_run_times": [_VP, ctypes.c_uint32, _VP, ctypes.POINTER(ctypes.c_uint32)],
        "ht_bytes_n": [_u64, _i, ctypes.POINTER(_u64)],
        "ht_create_n_at": [_u64, _i, ctypes.POINTER(ht_params), _VP, _u64, ctypes.POINTER(_VP)],
        "ht_buckets_for_bytes": [_u64, _i, ctypes.POINTER(ht_params), ctypes.POINTER(_u64)],
        "vss_line_divide": [ctypes.c_uint32, _VP, _u64, _VP, _VP],
        "reach_ctx_bytes_n": [_u64, _i, ctypes.c_uint32, ctypes.POINTER(_u64)],
        "reach_ctx_create_n_at": [_u64, _i, ctypes.c_uint32, ctypes.POINTER(ht_params), _VP, _u64,
                                  ctypes.POINTER(_VP)],
        "reach_ctx_buckets_for_bytes": [_u64, _i, ctypes.c_uint32, ctypes.POINTER(ht_params),
                                        ctypes.POINTER(_u64)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _st
    L.ht_status_string.argtypes = [_st]
    L.ht_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int, what: str):
    if status != HT_OK:
        raise HtError(status, what)


# ---------------------------------------------------------------------------
# Same-name thin wrappers (raw pointers as ints, streams as ints).
# ---------------------------------------------------------------------------

def ht_bytes(log2_buckets: int, state_words: int) -> int:
    out = _u64()
    _check(load().ht_bytes(log2_buckets, state_words, ctypes.byref(out)), "ht_bytes")
    return out.value


def ht_create(log2_buckets: int, state_words: int, params: ht_params | None = None) -> int:
    h = _VP()
    _check(load().ht_create(log2_buckets, state_words, ctypes.byref(params) if params else None,
                            ctypes.byref(h)), "ht_create")
    return h.value


def ht_create_at(log2_buckets, state_words, params, mem_dev: int, mem_bytes: int) -> int:
    h = _VP()
    _check(load().ht_create_at(log2_buckets, state_words, ctypes.byref(params) if params else None,
                               mem_dev, mem_bytes, ctypes.byref(h)), "ht_create_at")
    return h.value


def ht_destroy(h: int) -> int:
    return load().ht_destroy(h)


def ht_clear(h: int, stream: int = 0) -> int:
    return load().ht_clear(h, stream)


def ht_find_or_put(h: int, keys_dev: int, n: int, seen_dev: int, idx_dev: int, stream: int = 0) -> int:
    return load().ht_find_or_put(h, keys_dev, n, seen_dev, idx_dev, stream)


def ht_sync(h: int, stream: int = 0) -> int:
    return load().ht_sync(h, stream)


def ht_stats(h: int, stream: int = 0) -> ht_stats_t:
    s = ht_stats_t()
    _check(load().ht_stats(h, stream, ctypes.byref(s)), "ht_stats")
    return s


def ht_scan(h: int, stream: int = 0) -> tuple[int, int, int]:
    d, w, g = _u64(), _u64(), _u64()
    _check(load().ht_scan(h, stream, ctypes.byref(d), ctypes.byref(w), ctypes.byref(g)), "ht_scan")
    return d.value, w.value, g.value


def ht_gather(h: int, idx_dev: int, n: int, out_dev: int, stream: int = 0) -> int:
    return load().ht_gather(h, idx_dev, n, out_dev, stream)


def ht_arrays(h: int) -> tuple[int, int, int]:
    b, d, rw = _VP(), _VP(), ctypes.c_uint32()
    _check(load().ht_arrays(h, ctypes.byref(b), ctypes.byref(d), ctypes.byref(rw)), "ht_arrays")
    return b.value, d.value, rw.value


def ht_bytes_n(n_buckets: int, state_words: int) -> int:
    out = _u64()
    _check(load().ht_bytes_n(n_buckets, state_words, ctypes.byref(out)), "ht_bytes_n")
    return out.value


def ht_create_n_at(n_buckets, state_words, params, mem_dev: int, mem_bytes: int) -> int:
    h = _VP()
    _check(load().ht_create_n_at(n_buckets, state_words, ctypes.byref(params) if params else None,
                                 mem_dev, mem_bytes, ctypes.byref(h)), "ht_create_n_at")
    return h.value


def ht_buckets_for_bytes(nbytes: int, state_words: int, params: ht_params | None = None) -> int:
    out = _u64()
    _check(load().ht_buckets_for_bytes(nbytes, state_words, ctypes.byref(params) if params else None,
                                       ctypes.byref(out)), "ht_buckets_for_bytes")
    return out.value


def vss_line_divide(d: int, n) -> tuple[np.ndarray, np.ndarray]:
    """(n // d, n % d) through the library's invariant-divisor division (host)."""
    n = np.ascontiguousarray(n, dtype=np.uint64)
    q = np.empty_like(n)
    r = np.empty(n.shape, dtype=np.uint32)
    _check(load().vss_line_divide(d, n.ctypes.data, n.size, q.ctypes.data, r.ctypes.data),
           "vss_line_divide")
    return q, r


def reach_ctx_bytes_n(n_buckets: int, max_state_words: int, max_levels: int) -> int:
    out = _u64()
    _check(load().reach_ctx_bytes_n(n_buckets, max_state_words, max_levels, ctypes.byref(out)),
           "reach_ctx_bytes_n")
    return out.value


def reach_ctx_create_n_at(n_buckets, max_state_words, max_levels, params, mem_dev, mem_bytes) -> int:
    c = _VP()
    _check(load().reach_ctx_create_n_at(n_buckets, max_state_words, max_levels,
                                        ctypes.byref(params) if params else None, mem_dev, mem_bytes,
                                        ctypes.byref(c)), "reach_ctx_create_n_at")
    return c.value


def reach_ctx_buckets_for_bytes(nbytes: int, max_state_words: int, max_levels: int,
                                params: ht_params | None = None) -> int:
    out = _u64()
    _check(load().reach_ctx_buckets_for_bytes(nbytes, max_state_words, max_levels,
                                              ctypes.byref(params) if params else None,
                                              ctypes.byref(out)), "reach_ctx_buckets_for_bytes")
    return out.value


def reach_ctx_bytes(log2_buckets: int, max_state_words: int, max_levels: int) -> int:
    out = _u64()
    _check(load().reach_ctx_bytes(log2_buckets, max_state_words, max_levels, ctypes.byref(out)),
           "reach_ctx_bytes")
    return out.value


def reach_ctx_create_at(log2_buckets, max_state_words, max_levels, params, mem_dev, mem_bytes) -> int:
    c = _VP()
    _check(load().reach_ctx_create_at(log2_buckets, max_state_words, max_levels,
                                      ctypes.byref(params) if params else None, mem_dev, mem_bytes,
                                      ctypes.byref(c)), "reach_ctx_create_at")
    return c.value


def reach_ctx_create(log2_buckets, max_state_words, max_levels, params=None) -> int:
    c = _VP()
    _check(load().reach_ctx_create(log2_buckets, max_state_words, max_levels,
                                   ctypes.byref(params) if params else None, ctypes.byref(c)),
           "reach_ctx_create")
    return c.value


def reach_ctx_destroy(c: int) -> int:
    return load().reach_ctx_destroy(c)


class _ModelArgs:
    """Keeps the numpy arrays of a model alive while the C struct points at them."""

    def __init__(self, m):
        as32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        self.arrays = [as32(a) for a in (m.n_local, m.crit, m.edge_begin, m.edge_dst, m.guard_var,
                                         m.guard_val, m.upd_var, m.upd_val)]
        self.init = as32(m.init)
        p = [a.ctypes.data_as(_ip) for a in self.arrays]
        self.struct = reach_model(m.n_procs, m.n_shared, m.state_words, int(m.edge_dst.shape[0]), *p)


def reach_ctx_load(c: int, model, stream: int = 0) -> int:
    a = _ModelArgs(model)
    return load().reach_ctx_load(c, ctypes.byref(a.struct), a.init.ctypes.data, stream)


def reach_ctx_run(c: int, mode: int = REACH_PERSISTENT, stream: int = 0) -> int:
    return load().reach_ctx_run(c, mode, stream)


def reach_ctx_result(c: int, stream: int = 0, max_levels: int = 1 << 16):
    levels = np.zeros(max_levels, dtype=np.uint64)
    r = reach_result()
    st = load().reach_ctx_result(c, stream, levels.ctypes.data, max_levels, ctypes.byref(r))
    return st, r, levels[:min(r.n_levels, max_levels)].astype(np.int64)


def reach_ctx_last_timing(c: int) -> tuple[float, int]:
    ms, n = ctypes.c_float(), ctypes.c_uint32()
    _check(load().reach_ctx_last_timing(c, ctypes.byref(ms), ctypes.byref(n)), "reach_ctx_last_timing")
    return ms.value, n.value


def reach_ctx_level_ns(c: int, stream: int = 0, max_levels: int = 1 << 16) -> np.ndarray:
    out = np.zeros(max_levels, dtype=np.uint64)
    n = ctypes.c_uint32()
    _check(load().reach_ctx_level_ns(c, stream, out.ctypes.data, max_levels, ctypes.byref(n)),
           "reach_ctx_level_ns")
    return out[:n.value].astype(np.int64)


def reach_ctx_table(c: int) -> int:
    t = _VP()
    _check(load().reach_ctx_table(c, ctypes.byref(t)), "reach_ctx_table")
    return t.value


def reach(c: int, model, mode: int = REACH_PERSISTENT, stream: int = 0, max_levels: int = 1 << 16):
    a = _ModelArgs(model)
    levels = np.zeros(max_levels, dtype=np.uint64)
    r = reach_result()
    st = load().reach(c, ctypes.byref(a.struct), a.init.ctypes.data, mode, stream,
                      levels.ctypes.data, max_levels, ctypes.byref(r))
    return st, r, levels[:min(r.n_levels, max_levels)].astype(np.int64)


def vss_gen_keys(seed, n_ids, call_begin, n_calls, zipf_dev, state_words, keys_dev, stream=0) -> int:
    return load().vss_gen_keys(seed, n_ids, call_begin, n_calls, zipf_dev, state_words, keys_dev, stream)


def ht_find_or_put_stream(h, seed, n_ids, call_begin, n_calls, zipf_dev, result_dev, stream=0) -> int:
    return load().ht_find_or_put_stream(h, seed, n_ids, call_begin, n_calls, zipf_dev, result_dev,
                                        stream)


def vss_probe_random(buf_dev: int, nbytes: int, n_access: int, mode: int, stream: int = 0) -> float:
    ms = ctypes.c_float()
    _check(load().vss_probe_random(buf_dev, nbytes, n_access, mode, stream, ctypes.byref(ms)),
           "vss_probe_random")
    return ms.value


def vss_probe_random_cfg(buf_dev: int, nbytes: int, n_access: int, mode: int, inflight: int,
                         blocks_per_sm: int, threads: int, stream: int = 0) -> float:
    ms = ctypes.c_float()
    _check(load().vss_probe_random_cfg(buf_dev, nbytes, n_access, mode, inflight, blocks_per_sm,
                                       threads, stream, ctypes.byref(ms)), "vss_probe_random_cfg")
    return ms.value


PROBE_MODES = {0: "read 32 B", 1: "read 64 B", 2: "write 32 B", 3: "atomic 32-bit",
               4: "CAS 32-bit", 5: "CAS 16-bit", 6: "store 32-bit", 7: "store 16-bit",
               8: "read 4 B of a 32 B sector", 9: "read 64 B by 2 lanes", 10: "read 128 B by 4 lanes",
               11: "read 64 B by one bulk copy", 12: "write 64 B by one bulk copy"}

# Probe shapes swept for each mode: (accesses in flight per thread, blocks per
# SM, threads per block).  Reads hold their data in registers, so their
# resident blocks per SM fall as the in-flight count grows; the shapes keep
# several thousand requests in flight per SM in every case.
PROBE_SHAPES = {
    0: [(i, b, t) for i in (2, 4, 8, 16) for b in (8, 32) for t in (128, 256)],
    1: [(i, b, t) for i in (2, 4, 8) for b in (8, 32) for t in (128, 256)],
    8: [(i, b, t) for i in (4, 8, 16, 32, 64) for b in (8, 32) for t in (128, 256)],
    11: [(i, b, t) for i in (1, 2, 4, 8) for b in (8, 32) for t in (128, 256)],
    12: [(i, b, t) for i in (1, 2, 4, 8) for b in (8, 32) for t in (128, 256)],
}
DEFAULT_WRITE_SHAPES = [(i, b, 256) for i in (4, 8, 16) for b in (8, 32)]


def probe_sweep(gib: float = 16, n_access: int = 1 << 28, device="cuda", modes=(0, 1, 2, 3),
                reps: int = 3, shapes: dict | None = None) -> list:
    """Random accesses per second of every (mode, shape) in the sweep: a list
    of {"mode", "inflight", "blocks_per_sm", "threads", "per_s"} (best of reps)."""
    torch = _torch()
    nbytes = int(gib * (1 << 30)) // 256 * 256
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    ptr = (buf.data_ptr() + 255) // 256 * 256
    rows = []
    for mode in modes:
        for (inf, bps, thr) in (shapes or PROBE_SHAPES).get(mode, DEFAULT_WRITE_SHAPES):
            vss_probe_random_cfg(ptr, nbytes, n_access // 8, mode, inf, bps, thr, current_stream())
            ms = min(vss_probe_random_cfg(ptr, nbytes, n_access, mode, inf, bps, thr, current_stream())
                     for _ in range(reps))
            rows.append({"mode": mode, "inflight": inf, "blocks_per_sm": bps, "threads": thr,
                         "per_s": n_access / (ms / 1e3)})
    del buf
    torch.cuda.empty_cache()  # hand the probe buffer back to the driver
    return rows


def random_access_rates(gib: float = 16, n_access: int = 1 << 28, device="cuda",
                        modes=(0, 1, 2, 3), sweep: bool = True) -> dict:
    """Random accesses per second for each probe mode over a `gib` GiB buffer:
    the best rate over the probe shapes of PROBE_SHAPES (the plateau) when
    sweep is set, else the fixed default shape."""
    if sweep:
        rows = probe_sweep(gib, n_access, device, modes)
        return {m: max(r["per_s"] for r in rows if r["mode"] == m) for m in modes}
    torch = _torch()
    nbytes = int(gib * (1 << 30)) // 256 * 256
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    ptr = (buf.data_ptr() + 255) // 256 * 256
    out = {}
    for mode in modes:
        vss_probe_random(ptr, nbytes, n_access // 8, mode, current_stream())  # warm-up
        ms = min(vss_probe_random(ptr, nbytes, n_access, mode, current_stream()) for _ in range(3))
        out[mode] = n_access / (ms / 1e3)
    del buf
    torch.cuda.empty_cache()
    return out


def reach_noalloc(model, log2_buckets: int, params: ht_params | None = None, stream: int = 0,
                  max_levels: int = 4096):
    """reach() without device allocation (fixed 32 MiB scratch array inside the
    library); returns (status, reach_result, level sizes)."""
    a = _ModelArgs(model)
    levels = np.zeros(max_levels, dtype=np.uint64)
    r = reach_result()
    st = load().reach_noalloc(ctypes.byref(a.struct), a.init.ctypes.data, log2_buckets,
                              ctypes.byref(params) if params else None, stream, levels.ctypes.data,
                              max_levels, ctypes.byref(r))
    return st, r, levels[:min(r.n_levels, max_levels)].astype(np.int64)


# ---------------------------------------------------------------------------
# Torch-backed convenience layer.
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def current_stream() -> int:
    return _torch().cuda.current_stream().cuda_stream


def make_params(**kw) -> ht_params:
    p = ht_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Table:
    """A find-or-put table whose device memory is a torch uint8 tensor."""

    def __init__(self, log2_buckets: int | None, state_words: int, device="cuda",
                 n_buckets: int | None = None, **params):
        """2^log2_buckets buckets, or exactly n_buckets (log2_buckets None; any
        multiple of the line length, see ht_create_n_at)."""
        torch = _torch()
        if (log2_buckets is None) == (n_buckets is None):
            raise ValueError("give exactly one of log2_buckets and n_buckets")
        self.n_buckets = n_buckets if n_buckets is not None else 1 << log2_buckets
        self.log2_buckets, self.state_words = log2_buckets, state_words
        self.params = make_params(**params)
        nbytes = ht_bytes_n(self.n_buckets, state_words)
        self.mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.mem.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.handle = ht_create_n_at(self.n_buckets, state_words, self.params, aligned, nbytes)

    def close(self):
        if self.handle:
            ht_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self):
        _check(ht_clear(self.handle, current_stream()), "ht_clear")

    def find_or_put(self, keys, want_idx: bool = True):
        """keys: int32 CUDA tensor [n, state_words]. Returns (seen uint8, idx int32)."""
        torch = _torch()
        assert keys.is_cuda and keys.dtype == torch.int32 and keys.dim() == 2
        assert keys.shape[1] == self.state_words and keys.is_contiguous()
        n = keys.shape[0]
        seen = torch.empty(n, dtype=torch.uint8, device=keys.device)
        idx = torch.empty(n, dtype=torch.int32, device=keys.device) if want_idx else None
        _check(ht_find_or_put(self.handle, keys.data_ptr(), n, seen.data_ptr(),
                              idx.data_ptr() if idx is not None else 0, current_stream()),
               "ht_find_or_put")
        return seen, idx

    def find_or_put_stream(self, seed: int, n_ids: int, call_begin: int, n_calls: int,
                           zipf_table=None, sync: bool = True):
        """Fused generator + find-or-put over calls [call_begin, call_begin+n_calls)
        of the fill with n_ids keys; returns (new keys, digest of the stored keys)."""
        torch = _torch()
        zt = self._zipf_dev(zipf_table)
        res = torch.zeros(2, dtype=torch.int64, device=self.mem.device)
        _check(ht_find_or_put_stream(self.handle, seed, n_ids, call_begin, n_calls,
                                     zt.data_ptr() if zt is not None else 0, res.data_ptr(),
                                     current_stream()), "ht_find_or_put_stream")
        if not sync:
            return res
        v = res.cpu().numpy().view(np.uint64)
        return int(v[0]), int(v[1])

    def _zipf_dev(self, zipf_table):
        if zipf_table is None:
            return None
        torch = _torch()
        key = id(zipf_table)
        if getattr(self, "_zipf_key", None) != key:
            self._zipf = torch.from_numpy(np.ascontiguousarray(zipf_table, dtype=np.uint32).view(np.int32)).to(self.mem.device)
            self._zipf_key = key
        return self._zipf

    def gen_keys(self, seed: int, n_ids: int, call_begin: int, n_calls: int, zipf_table=None):
        """The keys of calls [call_begin, call_begin+n_calls) as an int32 CUDA tensor."""
        torch = _torch()
        zt = self._zipf_dev(zipf_table)
        out = torch.empty((n_calls, self.state_words), dtype=torch.int32, device=self.mem.device)
        _check(vss_gen_keys(seed, n_ids, call_begin, n_calls, zt.data_ptr() if zt is not None else 0,
                            self.state_words, out.data_ptr(), current_stream()), "vss_gen_keys")
        return out

    def sync(self) -> int:
        return ht_sync(self.handle, current_stream())

    def stats(self) -> ht_stats_t:
        return ht_stats(self.handle, current_stream())

    def scan(self):
        return ht_scan(self.handle, current_stream())

    def gather(self, idx):
        torch = _torch()
        out = torch.empty((idx.shape[0], self.state_words), dtype=torch.int32, device=idx.device)
        _check(ht_gather(self.handle, idx.data_ptr(), idx.shape[0], out.data_ptr(), current_stream()),
               "ht_gather")
        return out

    def arrays(self):
        """(bucket words as an int32 tensor, or int16 for 16-bit buckets; data
        int32 tensor [nb, row_words])."""
        torch = _torch()
        b, d, rw = ht_arrays(self.handle)
        nb = self.n_buckets
        base = self.mem.data_ptr()
        if self.params.bucket_bits == 16:
            buckets = self.mem[b - base:b - base + 2 * nb].view(torch.int16)
        else:
            buckets = self.mem[b - base:b - base + 4 * nb].view(torch.int32)
        data = self.mem[d - base:d - base + 4 * nb * rw].view(torch.int32).view(nb, rw)
        return buckets, data


@dataclass
class ReachOutput:
    states: int
    transitions: int
    deadlocks: int
    digest: int
    level_sizes: list
    busy_waits: int
    rehashes: int
    status: int


class ReachContext:
    """Device-resident reachability context (table + frontiers), memory from torch."""

    def __init__(self, log2_buckets: int | None, max_state_words: int, max_levels: int = 1 << 14,
                 device="cuda", n_buckets: int | None = None, **params):
        """2^log2_buckets buckets, or exactly n_buckets (log2_buckets None)."""
        torch = _torch()
        if (log2_buckets is None) == (n_buckets is None):
            raise ValueError("give exactly one of log2_buckets and n_buckets")
        self.n_buckets = n_buckets if n_buckets is not None else 1 << log2_buckets
        self.log2_buckets, self.max_state_words, self.max_levels = log2_buckets, max_state_words, max_levels
        self.params = make_params(**params)
        nbytes = reach_ctx_bytes_n(self.n_buckets, max_state_words, max_levels)
        self.mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        aligned = (self.mem.data_ptr() + 255) // 256 * 256
        self.handle = reach_ctx_create_n_at(self.n_buckets, max_state_words, max_levels, self.params,
                                            aligned, nbytes)

    def close(self):
        if self.handle:
            reach_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, model):
        _check(reach_ctx_load(self.handle, model, current_stream()), "reach_ctx_load")
        self._W = model.state_words

    def run(self, mode: int = REACH_PERSISTENT):
        _check(reach_ctx_run(self.handle, mode, current_stream()), "reach_ctx_run")

    def result(self, raise_on_error: bool = True) -> ReachOutput:
        st, r, levels = reach_ctx_result(self.handle, current_stream(), self.max_levels)
        if raise_on_error:
            _check(st, "reach_ctx_result")
        return ReachOutput(int(r.states), int(r.transitions), int(r.deadlocks), int(r.digest),
                           [int(x) for x in levels], int(r.busy_waits), int(r.rehashes), int(st))

    def reach(self, model, mode: int = REACH_PERSISTENT, raise_on_error: bool = True) -> ReachOutput:
        st, r, levels = reach(self.handle, model, mode, current_stream(), self.max_levels)
        self._W = model.state_words
        if raise_on_error:
            _check(st, "reach")
        return ReachOutput(int(r.states), int(r.transitions), int(r.deadlocks), int(r.digest),
                           [int(x) for x in levels], int(r.busy_waits), int(r.rehashes), int(st))

    def last_timing(self) -> tuple[float, int]:
        """(device ms of the last run's expansion kernels, kernels launched)."""
        return reach_ctx_last_timing(self.handle)

    def deadlock_trace(self, max_len: int = 1 << 14):
        """(level, path rows init..deadlock) of the last REACH_TRACE run, or (None, empty)."""
        W = getattr(self, "_W", self.max_state_words)
        buf = np.zeros((max_len, W), dtype=np.int32)
        n, lv = ctypes.c_uint32(), ctypes.c_uint32()
        _check(load().reach_ctx_deadlock_trace(self.handle, current_stream(), buf.ctypes.data, max_len,
                                               ctypes.byref(n), ctypes.byref(lv)), "reach_ctx_deadlock_trace")
        if n.value == 0:
            return None, buf[:0]
        return int(lv.value), buf[:n.value]

    def run_times(self, n: int) -> np.ndarray:
        """Kernel device times (ms) of the last n runs (at most 64), oldest first."""
        out = np.zeros(n, dtype=np.float32)
        got = ctypes.c_uint32()
        _check(load().reach_ctx_run_times(self.handle, n, out.ctypes.data, ctypes.byref(got)),
               "reach_ctx_run_times")
        return out[:got.value]

    def level_ns(self) -> np.ndarray:
        """Device timestamps (ns) of the level starts of the last persistent run."""
        return reach_ctx_level_ns(self.handle, current_stream(), self.max_levels)

    def table_handle(self) -> int:
        return reach_ctx_table(self.handle)

    def scan(self):
        return ht_scan(self.table_handle(), current_stream())


# ---------------------------------------------------------------------------
# Owner-partitioned reachability (static partitioning, K owners on one GPU).
# ---------------------------------------------------------------------------

def part_reach_bytes(n_parts: int, log2_buckets_part: int, max_state_words: int,
                     exchange_rows: int) -> int:
    out = _u64()
    _check(load().part_reach_bytes(n_parts, log2_buckets_part, max_state_words, exchange_rows,
                                   ctypes.byref(out)), "part_reach_bytes")
    return out.value


class PartReach:
    """n_parts owner partitions of 2^log2_buckets_part buckets each on one
    GPU (part_reach_*), device memory from a torch tensor."""

    def __init__(self, n_parts: int, log2_buckets_part: int, max_state_words: int,
                 exchange_rows: int = 1 << 20, max_levels: int = 1 << 14, device="cuda", **params):
        torch = _torch()
        self.n_parts, self.max_levels = n_parts, max_levels
        self.params = make_params(**params)
        nbytes = part_reach_bytes(n_parts, log2_buckets_part, max_state_words, exchange_rows)
        self.mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        aligned = (self.mem.data_ptr() + 255) // 256 * 256
        h = _VP()
        _check(load().part_reach_create_at(n_parts, log2_buckets_part, max_state_words, exchange_rows,
                                           ctypes.byref(self.params), aligned, nbytes, ctypes.byref(h)),
               "part_reach_create_at")
        self.handle = h.value

    def close(self):
        if self.handle:
            load().part_reach_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, model, raise_on_error: bool = True):
        """(ReachOutput, states per partition, successors exchanged between partitions)."""
        a = _ModelArgs(model)
        levels = np.zeros(self.max_levels, dtype=np.uint64)
        parts = np.zeros(self.n_parts, dtype=np.uint64)
        ex = _u64()
        r = reach_result()
        st = load().part_reach_run(self.handle, ctypes.byref(a.struct), a.init.ctypes.data,
                                   current_stream(), levels.ctypes.data, self.max_levels,
                                   ctypes.byref(r), parts.ctypes.data, ctypes.byref(ex))
        if raise_on_error:
            _check(st, "part_reach_run")
        lv = [int(x) for x in levels[:min(r.n_levels, self.max_levels)]]
        out = ReachOutput(int(r.states), int(r.transitions), int(r.deadlocks), int(r.digest), lv,
                          int(r.busy_waits), int(r.rehashes), int(st))
        return out, [int(x) for x in parts], int(ex.value)

    def last_exchange(self):
        """(counts [n, n], inbox segment offsets [n, n], inbox starts [n + 1]) of the last chunk."""
        K = self.n_parts
        counts = np.zeros((K, K), dtype=np.uint32)
        seg = np.zeros((K, K), dtype=np.uint32)
        begin = np.zeros(K + 1, dtype=np.uint32)
        _check(load().part_reach_last_exchange(self.handle, counts.ctypes.data, seg.ctypes.data,
                                               begin.ctypes.data), "part_reach_last_exchange")
        return counts, seg, begin


# ---------------------------------------------------------------------------
# Batched reachability (many models, one persistent launch).
# ---------------------------------------------------------------------------

def generation_bytes(log2_buckets: int, state_words: int) -> int:
    """Bytes of one table generation: buckets, data rows and two frontiers."""
    nb = 1 << log2_buckets
    nv = (state_words + 3) // 4
    up = lambda x: (x + 255) // 256 * 256
    return up(4 * nb) + 3 * up(16 * nv * nb)


def default_pool_bytes(models, log2_initial=None) -> int:
    """Pool for the initial tables plus growth up to 50% load of each model's
    state bound (product of local state counts when there are no shared
    variables; otherwise 2^22 states is assumed)."""
    total = 0
    for i, m in enumerate(models):
        bound = int(np.prod(np.asarray(m.n_local, dtype=np.float64))) if m.n_shared == 0 else 1 << 22
        final = max(10, int(np.ceil(np.log2(max(bound, 1) / 0.5))))
        init = (log2_initial[i] if log2_initial is not None and log2_initial[i] else min(final, 16))
        g = generation_bytes(init, m.state_words)
        lg = init
        while lg < final:
            lg += 1
            g += generation_bytes(lg, m.state_words)
        total += g
    return total + (64 << 20)


class ReachBatch:
    """Many independent models expanded by one persistent kernel (optionally
    replayed as a CUDA graph); device memory from a torch tensor."""

    def __init__(self, models, log2_initial=None, max_levels: int = 4096, pool_bytes: int | None = None,
                 device="cuda", **params):
        torch = _torch()
        self.models = list(models)
        self.n = len(self.models)
        self.max_levels = max_levels
        self.params = make_params(**params)
        self._args = [_ModelArgs(m) for m in self.models]
        self._structs = (reach_model * self.n)(*[a.struct for a in self._args])
        self._inits = (ctypes.c_void_p * self.n)(*[a.init.ctypes.data for a in self._args])
        self._log2 = None
        if log2_initial is not None:
            self._log2 = np.ascontiguousarray(log2_initial, dtype=np.int32)
        self.pool_bytes = pool_bytes or default_pool_bytes(self.models, log2_initial)
        out = _u64()
        _check(load().reach_batch_bytes(ctypes.byref(self._structs), ctypes.byref(self._inits), self.n,
                                        max_levels, self.pool_bytes, ctypes.byref(out)), "reach_batch_bytes")
        self.mem = torch.empty(out.value + 256, dtype=torch.uint8, device=device)
        aligned = (self.mem.data_ptr() + 255) // 256 * 256
        h = _VP()
        _check(load().reach_batch_create_at(ctypes.byref(self._structs), ctypes.byref(self._inits), self.n,
                                            self._log2.ctypes.data if self._log2 is not None else None,
                                            max_levels, self.pool_bytes, ctypes.byref(self.params),
                                            aligned, out.value, ctypes.byref(h)), "reach_batch_create_at")
        self.handle = h.value

    def close(self):
        if self.handle:
            load().reach_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, use_graph: bool = True):
        _check(load().reach_batch_run(self.handle, int(use_graph), current_stream()), "reach_batch_run")

    def last_timing(self) -> float:
        ms = ctypes.c_float()
        _check(load().reach_batch_last_timing(self.handle, ctypes.byref(ms)), "reach_batch_last_timing")
        return ms.value

    def results(self):
        """(list of ReachOutput, grows per model, overall status)."""
        outs = (reach_result * self.n)()
        levels = np.zeros(self.n * self.max_levels, dtype=np.uint64)
        grows = np.zeros(self.n, dtype=np.uint32)
        st = load().reach_batch_results(self.handle, current_stream(), ctypes.byref(outs),
                                        levels.ctypes.data, grows.ctypes.data)
        res = []
        for i in range(self.n):
            r = outs[i]
            lv = levels[i * self.max_levels:i * self.max_levels + min(r.n_levels, self.max_levels)]
            res.append(ReachOutput(int(r.states), int(r.transitions), int(r.deadlocks), int(r.digest),
                                   [int(x) for x in lv], int(r.busy_waits), int(r.rehashes), int(r.status)))
        return res, [int(x) for x in grows], int(st)


# ---------------------------------------------------------------------------
# Serving (continuous batching of reachability jobs).
# ---------------------------------------------------------------------------

class serve_done_t(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_uint64), ("result", reach_result), ("grows", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


@dataclass
class ServedJob:
    job_id: int
    result: ReachOutput
    submit_s: float
    admit_s: float
    done_s: float

    @property
    def latency_s(self) -> float:
        return self.done_s - self.submit_s


class Server:
    """Reachability request loop: jobs are admitted by HBM budget into slots of
    one persistent kernel (continuous batching); arena memory from torch."""

    def __init__(self, budget_bytes: int, n_slots: int = 64, max_levels: int = 4096, device="cuda",
                 **params):
        torch = _torch()
        self.max_levels = max_levels
        self.params = make_params(**params)
        out = _u64()
        _check(load().serve_bytes(budget_bytes, n_slots, max_levels, ctypes.byref(out)), "serve_bytes")
        self.mem = torch.empty(out.value + 256, dtype=torch.uint8, device=device)
        aligned = (self.mem.data_ptr() + 255) // 256 * 256
        h = _VP()
        _check(load().serve_open_at(aligned, out.value, n_slots, max_levels, ctypes.byref(self.params),
                                    ctypes.byref(h)), "serve_open_at")
        self.handle = h.value
        self._keep = {}

    def submit(self, model, log2_buckets: int = 0) -> int:
        a = _ModelArgs(model)
        jid = _u64()
        _check(load().serve_submit(self.handle, ctypes.byref(a.struct), a.init.ctypes.data, log2_buckets,
                                   ctypes.byref(jid)), "serve_submit")
        return jid.value

    def poll(self, max_done: int = 256, want_levels: bool = True):
        done = (serve_done_t * max_done)()
        n = ctypes.c_uint32()
        levels = np.zeros(max_done * self.max_levels, dtype=np.uint64) if want_levels else None
        _check(load().serve_poll(self.handle, ctypes.byref(done), max_done, ctypes.byref(n),
                                 levels.ctypes.data if levels is not None else None), "serve_poll")
        out = []
        for i in range(n.value):
            d = done[i]
            r = d.result
            lv = []
            if levels is not None:
                lv = [int(x) for x in levels[i * self.max_levels:i * self.max_levels + min(r.n_levels, self.max_levels)]]
            out.append(ServedJob(int(d.job_id), ReachOutput(int(r.states), int(r.transitions), int(r.deadlocks),
                                                            int(r.digest), lv, int(r.busy_waits), int(r.rehashes),
                                                            int(r.status)), d.submit_s, d.admit_s, d.done_s))
        return out

    def status(self):
        q, r, f, k = ctypes.c_uint32(), ctypes.c_uint32(), _u64(), _u64()
        _check(load().serve_status(self.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f),
                                   ctypes.byref(k)), "serve_status")
        return {"queued": q.value, "running": r.value, "free_bytes": f.value, "kernel_launches": k.value}

    def close(self):
        if self.handle:
            _check(load().serve_close(self.handle), "serve_close")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
