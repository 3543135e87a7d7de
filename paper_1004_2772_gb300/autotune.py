"""Autotuner for the store's layout and probing parameters.

The paper leaves several "sensitive performance parameters" to the implementer
(Abstract and Sec. 1: bucket size, cache-line size, data layout, probing
sequence).  Here the tunable ones are

    line_buckets   walk length: buckets walked per line before rehashing (8,
                   16, 32: a 32-, 64- or 128-byte line, read one 32-byte
                   sector at a time)
    bucket_bits    bucket width: 32 (31-bit memo) or 16 (15-bit memo, half the
                   bucket array, lines of 16 or 32 buckets)
    group_lanes    lanes per key: 1 (a thread walks the line sector by sector)
                   or 2, 4, 8 (a sub-warp group loads a line of 4G buckets)
    dedup          merge equal keys inside a warp before probing (hot keys)
    block_threads  threads per block of the batch / expansion kernels
    rehash         rehash sequence after a full line: double hashing (0) or
                   the next line (1)
    max_rehash     lines probed before a key gives up (0 = the default bound)
    log2_buckets   table size for the same states (reachability): the load factor

The search is staged: first the layout (walk length, bucket width, lanes,
dedup, block size), then the probe sequence (rehash rule, rehash bound) on the
best layout, then, for reachability, the table size.  Every candidate must
give identical results (number of keys stored and the digest of the stored set
for the key-stream benchmark; states, transitions, deadlocks, level sizes and
digest for reachability); a candidate that disagrees is an error, not a slower
choice.  A candidate that cannot finish (a rehash bound too small for the
load, a table too small for the states: HT_ERR_FULL) is recorded as not
admissible and never chosen.  Choices are cached in a JSON file keyed by the
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
REACH_SPACE = {"line_buckets": (8, 16, 32), "bucket_bits": (32, 16), "group_lanes": (1, 2, 4, 8),
               "block_threads": (128, 256)}
# probe sequence, tried on the best layout
PROBE_SPACE = {"rehash": (0, 1), "max_rehash": (0, 256, 16)}
REACH_PROBE_SPACE = {"rehash": (0, 1)}
# extra doublings of the reachability table tried last (lower load factors)
LOAD_STEPS = (0, 1)

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
    """Device ms of one fill (2 * n_ids calls of the key stream), median of
    reps, and (keys stored, digest), or None when the fill failed."""
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
        if tab.stats().error:
            return float(np.median(ms)), None
        v = res.cpu().numpy().view(np.uint64)
        out = (int(v[0]), int(v[1]))
    return float(np.median(ms)), out


def _check(res, ref, cand):
    """Reference result of the first admissible candidate; later ones must agree."""
    if ref is None:
        return res
    if res != ref:
        raise RuntimeError(f"parameters {cand} changed the result")
    return ref


def tune_table(log2_buckets: int, load_factor: float, dist: str = "uniform", state_words: int = 16,
               seed: int = 1, space=None, probe_space=None, reps: int = 3,
               cache_path: str | None = DEFAULT_CACHE, verbose: bool = False):
    """Best table parameters for one fill of 2^log2 * load_factor keys (half of
    the calls repeat a key, uniformly or Zipf(1.1))."""
    from . import synth
    key = f"table-W{state_words}-n{log2_buckets}-lf{load_factor}-{dist}"
    cache = _load_cache(cache_path) if cache_path else {}
    if key in cache and space is None and probe_space is None:
        return cache[key]
    n_ids = int(load_factor * (1 << log2_buckets))
    zipf = synth.zipf_table(n_ids) if dist == "zipf" else None
    rows, ref = [], None

    def trial(cand, stage):
        nonlocal ref
        tab = B.Table(log2_buckets, state_words, **cand)
        ms, res = time_fill(tab, seed, n_ids, zipf, reps)
        tab.close()
        ok = res is not None
        if ok:
            ref = _check(res, ref, cand)
        rows.append({"params": cand, "stage": stage, "ms": ms, "admissible": ok,
                     "ops_per_s": 2 * n_ids / (ms / 1e3)})
        if verbose:
            print(key, stage, cand, f"{ms:.3f} ms", "" if ok else "(not admissible)", flush=True)

    for cand in _candidates(space or TABLE_SPACE):
        trial(cand, "layout")
    best = _best(rows)
    for probe in _candidates(probe_space or PROBE_SPACE):
        if all(v == 0 for v in probe.values()):
            continue  # the defaults: the layout stage measured them
        trial({**best["params"], **probe}, "probe")
    best = _best(rows)
    entry = {"best": best["params"], "ms": best["ms"], "ops_per_s": best["ops_per_s"],
             "n_new": ref[0], "digest": f"{ref[1]:#018x}", "all": rows, "when": time.time()}
    if cache_path:
        cache[key] = entry
        _save_cache(cache_path, cache)
    return entry


def _best(rows):
    ok = [r for r in rows if r["admissible"]]
    if not ok:
        raise RuntimeError("no admissible candidate")
    return min(ok, key=lambda r: r["ms"])


def tune_reach(model, log2_buckets: int, space=None, probe_space=None, load_steps=None,
               reps: int = 3, cache_path: str | None = DEFAULT_CACHE, verbose: bool = False):
    """Best reachability parameters for one model (persistent driver): the
    layout at 2^log2_buckets buckets, then the rehash rule, then the table size
    (log2_buckets + each of load_steps, i.e. lower load factors)."""
    key = f"reach-{model.name}-n{log2_buckets}"
    cache = _load_cache(cache_path) if cache_path else {}
    if key in cache and space is None and probe_space is None and load_steps is None:
        return cache[key]
    rows, ref = [], None

    def trial(cand, stage):
        nonlocal ref
        cand = dict(cand)
        lg = cand.pop("log2_buckets", log2_buckets)
        ctx = B.ReachContext(lg, model.state_words, max_levels=1 << 14, **cand)
        ctx.load(model)
        ms = []
        for _ in range(reps):
            ctx.run(B.REACH_PERSISTENT)
            ms.append(ctx.last_timing()[0])
        r = ctx.result(raise_on_error=False)
        ctx.close()
        ok = r.status == 0
        if ok:
            ref = _check((r.states, r.transitions, r.deadlocks, r.digest, tuple(r.level_sizes)), ref,
                         cand)
        rows.append({"params": {**cand, "log2_buckets": lg}, "stage": stage,
                     "ms": float(np.median(ms)), "admissible": ok})
        if verbose:
            print(key, stage, cand, lg, f"{np.median(ms):.3f} ms", flush=True)

    for cand in _candidates(space or REACH_SPACE):
        trial(cand, "layout")
    best = _best(rows)["params"]
    for probe in _candidates(probe_space or REACH_PROBE_SPACE):
        if all(v == 0 for v in probe.values()):
            continue
        trial({**best, **probe}, "probe")
    best = _best(rows)["params"]
    for d in (LOAD_STEPS if load_steps is None else load_steps):
        if d == 0:
            continue
        trial({**best, "log2_buckets": log2_buckets + d}, "load")
    b = _best(rows)
    entry = {"best": b["params"], "ms": b["ms"], "states": ref[0], "transitions": ref[1],
             "deadlocks": ref[2], "digest": f"{ref[3]:#018x}", "level_sizes": list(ref[4]),
             "all": rows, "when": time.time()}
    if cache_path:
        cache[key] = entry
        _save_cache(cache_path, cache)
    return entry
