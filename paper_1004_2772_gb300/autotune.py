"""Autotuner for the store's layout parameters.

The paper leaves several "sensitive performance parameters" to the implementer
(Section 1: bucket size, cache-line size, data layout, probing sequence).  Here
the tunable ones are

    line_buckets   buckets walked per line before rehashing (8, 16, 32: a 32-,
                   64- or 128-byte line, read one 32-byte sector at a time)
    bucket_bits    bucket width: 32 (31-bit memo) or 16 (15-bit memo, half the
                   bucket array, lines of 16 or 32 buckets)
    group_lanes    lanes per key: 1 (a thread walks the line sector by sector)
                   or 2, 4, 8 (a sub-warp group loads a line of 4G buckets)
    dedup          merge equal keys inside a warp before probing (hot keys)
    block_threads  threads per block of the batch / expansion kernels
    log2_buckets   table size for a given number of keys (the load factor)

Every candidate must give identical results (number of keys stored and the
digest of the stored set for the key-stream benchmark; states, transitions,
level sizes and digest for reachability); a candidate that disagrees is an
error, not a slower choice.  Choices are cached in a JSON file keyed by the
workload shape.  The hash family is fixed by the implementation.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from . import binding as B

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1004_2772_gb300_autotune.json")

TABLE_SPACE = {"line_buckets": (8, 16, 32), "bucket_bits": (32, 16), "dedup": (0, 1),
               "group_lanes": (1, 2, 4, 8), "block_threads": (128, 256)}
REACH_SPACE = {"line_buckets": (8, 16, 32), "bucket_bits": (32, 16), "block_threads": (128, 256)}

# line lengths each bucket width supports (a line is 1, 2 or 4 sectors of 32 bytes)
LINES_FOR_WIDTH = {32: (8, 16, 32), 16: (16, 32)}


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _candidates(space):
    keys = sorted(space)
    for vals in itertools.product(*(space[k] for k in keys)):
        cand = dict(zip(keys, vals))
        if cand.get("line_buckets", 0) not in LINES_FOR_WIDTH[cand.get("bucket_bits", 32)] + (0,):
            continue
        g = cand.get("group_lanes", 1)
        if g > 1 and (cand.get("line_buckets", 4 * g) != 4 * g or cand.get("bucket_bits", 32) != 32
                      or cand.get("dedup", 0)):
            continue  # a group reads one whole line of 4G 32-bit buckets
        yield cand


def time_fill(tab, seed, n_ids, zipf=None, reps=1):
    """Device ms of one fill (2 * n_ids calls of the key stream), median of reps."""
    import torch
    ms = []
    out = None
    for _ in range(reps):
        tab.clear()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = tab.find_or_put_stream(seed, n_ids, 0, 2 * n_ids, zipf, sync=False)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        v = res.cpu().numpy().view(np.uint64)
        out = (int(v[0]), int(v[1]))
    return float(np.median(ms)), out


def tune_table(log2_buckets: int, load_factor: float, dist: str = "uniform", state_words: int = 16,
               seed: int = 1, space=None, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
               verbose: bool = False):
    """Best table parameters for one fill of 2^log2 * load_factor keys (half of
    the calls repeat a key, uniformly or Zipf(1.1))."""
    from . import synth
    key = f"table-W{state_words}-n{log2_buckets}-lf{load_factor}-{dist}"
    cache = _load_cache(cache_path) if cache_path else {}
    if key in cache and space is None:
        return cache[key]
    n_ids = int(load_factor * (1 << log2_buckets))
    zipf = synth.zipf_table(n_ids) if dist == "zipf" else None
    rows, ref = [], None
    for cand in _candidates(space or TABLE_SPACE):
        tab = B.Table(log2_buckets, state_words, **cand)
        ms, res = time_fill(tab, seed, n_ids, zipf, reps)
        if ref is None:
            ref = res
        elif res != ref:
            raise RuntimeError(f"parameters {cand} changed the result: {res} != {ref}")
        rows.append({"params": cand, "ms": ms, "ops_per_s": 2 * n_ids / (ms / 1e3)})
        if verbose:
            print(key, cand, f"{ms:.3f} ms", flush=True)
        tab.close()
    best = min(rows, key=lambda r: r["ms"])
    entry = {"best": best["params"], "ms": best["ms"], "ops_per_s": best["ops_per_s"],
             "n_new": ref[0], "digest": f"{ref[1]:#018x}", "all": rows, "when": time.time()}
    if cache_path:
        cache[key] = entry
        _save_cache(cache_path, cache)
    return entry


def tune_reach(model, log2_buckets: int, space=None, reps: int = 3,
               cache_path: str | None = DEFAULT_CACHE, verbose: bool = False):
    """Best reachability parameters for one model (persistent driver)."""
    key = f"reach-{model.name}-n{log2_buckets}"
    cache = _load_cache(cache_path) if cache_path else {}
    if key in cache and space is None:
        return cache[key]
    rows, ref = [], None
    for cand in _candidates(space or REACH_SPACE):
        ctx = B.ReachContext(log2_buckets, model.state_words, max_levels=1 << 14, **cand)
        ctx.load(model)
        ms = []
        for _ in range(reps):
            ctx.run(B.REACH_PERSISTENT)
            ms.append(ctx.last_timing()[0])
        r = ctx.result()
        res = (r.states, r.transitions, r.deadlocks, r.digest, tuple(r.level_sizes))
        if ref is None:
            ref = res
        elif res != ref:
            raise RuntimeError(f"parameters {cand} changed the result")
        rows.append({"params": cand, "ms": float(np.median(ms))})
        if verbose:
            print(key, cand, f"{np.median(ms):.3f} ms", flush=True)
        ctx.close()
    best = min(rows, key=lambda r: r["ms"])
    entry = {"best": best["params"], "ms": best["ms"], "states": ref[0], "all": rows,
             "when": time.time()}
    if cache_path:
        cache[key] = entry
        _save_cache(cache_path, cache)
    return entry
