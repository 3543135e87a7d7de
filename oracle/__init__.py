"""CPU oracle for the visited-state store -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this package.  The product path (``paper_1004_2772_gb300``) never
imports it, and it never imports the product path: the two share nothing but
the seeded input generator ``paper_1004_2772_gb300.synth`` (random tables, no
method arithmetic), whose Model objects are plain numpy arrays.

The oracle itself is ``oracle.cpp``: single-threaded, std::unordered_set, strict
level-by-level BFS (Alg. "Reachability analysis"), and find-or-put over a key
stream in stream order (Section 3.1).  This module compiles it with g++ and
wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_libs: dict[int, ctypes.CDLL] = {}


def lib_path(plant: int = 0) -> str:
    return os.path.join(_BUILD, "liboracle.so" if plant == 0 else f"liboracle_plant{plant}.so")


def build(plant: int = 0, force: bool = False) -> str:
    """Compile oracle.cpp (plant > 0 builds a test variant with one planted mistake)."""
    out = lib_path(plant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-shared", "-fPIC", f"-DORACLE_PLANT={plant}", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_P = ctypes.c_void_p
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int32


def _load(plant: int = 0) -> ctypes.CDLL:
    if plant in _libs:
        return _libs[plant]
    lib = ctypes.CDLL(build(plant))
    lib.oracle_splitmix64.restype = _u64
    lib.oracle_splitmix64.argtypes = [_u64]
    lib.oracle_state_fingerprint.restype = _u64
    lib.oracle_state_fingerprint.argtypes = [_P, ctypes.c_int]
    lib.oracle_digest.restype = _u64
    lib.oracle_digest.argtypes = [_P, _u64, ctypes.c_int]
    lib.oracle_successors.restype = ctypes.c_int64
    lib.oracle_successors.argtypes = [ctypes.c_int] * 3 + [_P] * 9 + [_P, ctypes.c_int64]
    lib.oracle_reach.restype = ctypes.c_int
    lib.oracle_reach.argtypes = ([ctypes.c_int] * 3 + [_P] * 9 + [_u64, ctypes.c_uint32]
                                 + [_P] * 7 + [_P, _u64])
    lib.oracle_find_or_put_stream.restype = _u64
    lib.oracle_find_or_put_stream.argtypes = [_P, _u64, ctypes.c_int, _P, _P, _P]
    _libs[plant] = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _model_args(m):
    arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in
            (m.n_local, m.crit, m.edge_begin, m.edge_dst, m.guard_var, m.guard_val, m.upd_var,
             m.upd_val)]
    return arrs, [m.n_procs, m.n_shared, m.state_words] + [_ptr(a) for a in arrs]


def splitmix64(z: int, plant: int = 0) -> int:
    return int(_load(plant).oracle_splitmix64(z & ((1 << 64) - 1)))


def fingerprint(v, plant: int = 0) -> int:
    a = np.ascontiguousarray(v, dtype=np.int32)
    return int(_load(plant).oracle_state_fingerprint(_ptr(a), a.shape[0]))


def digest(states: np.ndarray, plant: int = 0) -> int:
    a = np.ascontiguousarray(states, dtype=np.int32)
    return int(_load(plant).oracle_digest(_ptr(a), a.shape[0], a.shape[1]))


def successors(m, v, plant: int = 0) -> np.ndarray:
    keep, args = _model_args(m)
    v = np.ascontiguousarray(v, dtype=np.int32)
    cap = 4096
    out = np.zeros((cap, m.state_words), dtype=np.int32)
    n = _load(plant).oracle_successors(*args, _ptr(v), _ptr(out), cap)
    assert n <= cap
    return out[:n].copy()


@dataclass
class ReachResult:
    states: int
    transitions: int
    deadlocks: int
    digest: int
    level_sizes: list
    truncated: bool
    state_list: np.ndarray | None = None


def reach(m, max_states: int = 1 << 62, max_levels: int = 1 << 16, keep_states: bool = False,
          plant: int = 0, keep_cap: int = 1 << 20) -> ReachResult:
    """Level-synchronous BFS from m.init; see oracle.cpp for the definitions."""
    keep, args = _model_args(m)
    init = np.ascontiguousarray(m.init, dtype=np.int32)
    levels = np.zeros(max_levels, dtype=np.uint64)
    o = [np.zeros(1, dtype=np.uint64) for _ in range(4)]
    nl = np.zeros(1, dtype=np.uint32)
    tr = np.zeros(1, dtype=np.int32)
    st = None
    cap = 0
    if keep_states:
        cap = min(max_states + 1, keep_cap)
        st = np.empty((cap, m.state_words), dtype=np.int32)
    _load(plant).oracle_reach(*args, _ptr(init), max_states, max_levels,
                              _ptr(o[0]), _ptr(o[1]), _ptr(o[2]), _ptr(o[3]), _ptr(levels),
                              _ptr(nl), _ptr(tr), _ptr(st) if st is not None else None, cap)
    n = int(o[0][0])
    return ReachResult(states=n, transitions=int(o[1][0]), deadlocks=int(o[2][0]),
                       digest=int(o[3][0]), level_sizes=[int(x) for x in levels[:int(nl[0])]],
                       truncated=bool(tr[0]),
                       state_list=st[:min(n, cap)].copy() if st is not None else None)


@dataclass
class StreamResult:
    n_new: int
    seen: np.ndarray
    first: np.ndarray
    digest: int


def find_or_put_stream(keys: np.ndarray, plant: int = 0) -> StreamResult:
    """find-or-put of each key in stream order (Section 3.1)."""
    k = np.ascontiguousarray(keys, dtype=np.int32)
    n, W = k.shape
    seen = np.zeros(n, dtype=np.uint8)
    first = np.zeros(n, dtype=np.uint64)
    d = np.zeros(1, dtype=np.uint64)
    n_new = _load(plant).oracle_find_or_put_stream(_ptr(k), n, W, _ptr(seen), _ptr(first), _ptr(d))
    return StreamResult(n_new=int(n_new), seen=seen, first=first, digest=int(d[0]))
