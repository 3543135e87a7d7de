"""The find-or-put protocol written as a model for reach() (test helper).

The paper checked its find-or-put algorithm by modelling it in PROMELA and
exploring it with SPIN, which found one bug about the write bit and the
memoised hash (Section 3.3).  Here the same protocol -- the one the CUDA table
runs -- is written in this project's own model encoding and explored by
reach() itself: every interleaving of T threads inserting keys into a line of
B buckets.

Processes are threads; shared variables are the B bucket words and the B data
words.  A bucket word is 0 (empty), 2m-1 (write, memo m) or 2m (done, memo m).
Thread t inserts key k_t whose memo is memo_t; its local states are, for each
bucket i in walk order,
    PROBE(i)  CAS empty -> write(memo)       (one atomic edge: guard b_i == 0, b_i := 2m-1)
              wait while write(memo)          (self-loop: guard b_i == 2m-1)
              done(memo) -> CMP(i)            (guard b_i == 2m)
              another memo -> next bucket     (guard b_i == that value)
    DATA(i)   d_i := k                        (the data write after the claim)
    PUB(i)    b_i := 2m                       (publish done)
    CMP(i)    d_i == k -> SEEN; d_i == another key with this memo -> next bucket
and the terminal states NEW, SEEN, FULL.  Keys that share a memo exercise the
data compare; equal keys exercise the claim race and the write-busy wait.

`broken="skip_write"` plants the classic mistake around the write bit: a
thread that meets its own memo still in the write state moves on to the next
bucket instead of waiting, which lets two threads insert the same key.
"""
from __future__ import annotations

import numpy as np

from paper_1004_2772_gb300 import synth

NEW, SEEN, FULL = "NEW", "SEEN", "FULL"


def protocol_model(keys, memos, n_buckets, broken: str | None = None):
    T, B = len(keys), n_buckets
    memo_vals = sorted(set(memos))
    bucket_vals = [0] + [v for m in memo_vals for v in (2 * m - 1, 2 * m)]
    key_vals = sorted(set(keys))
    # local state numbering per thread
    names = []
    for i in range(B):
        names += [("PROBE", i), ("DATA", i), ("PUB", i), ("CMP", i)]
    names += [(NEW, -1), (SEEN, -1), (FULL, -1)]
    idx = {n: j for j, n in enumerate(names)}
    bvar = lambda i: i          # shared variable index of bucket i
    dvar = lambda i: B + i      # shared variable index of data word i
    edges = []
    for t in range(T):
        k, m = keys[t], memos[t]
        wr, dn = 2 * m - 1, 2 * m
        et = []
        for (kind, i) in names:
            nxt = ("PROBE", i + 1) if i + 1 < B else (FULL, -1)
            if kind == "PROBE":
                es = [(idx[("DATA", i)], bvar(i), 0, bvar(i), wr)]
                if broken == "skip_write":
                    es.append((idx[nxt], bvar(i), wr, -1, 0))
                else:
                    es.append((idx[("PROBE", i)], bvar(i), wr, -1, 0))
                es.append((idx[("CMP", i)], bvar(i), dn, -1, 0))
                for v in bucket_vals:
                    if v not in (0, wr, dn):
                        es.append((idx[nxt], bvar(i), v, -1, 0))
            elif kind == "DATA":
                es = [(idx[("PUB", i)], -1, 0, dvar(i), k)]
            elif kind == "PUB":
                es = [(idx[(NEW, -1)], -1, 0, bvar(i), dn)]
            elif kind == "CMP":
                es = [(idx[(SEEN, -1)], dvar(i), k, -1, 0)]
                for k2 in key_vals:
                    if k2 != k:
                        es.append((idx[nxt], dvar(i), k2, -1, 0))
            else:
                es = []
            et.append(es)
        edges.append(et)
    n_local = [len(names)] * T
    init = [idx[("PROBE", 0)]] * T + [0] * (2 * B)
    m = synth.build_model(f"protocol-T{T}-B{B}-{broken or 'ok'}", n_local, edges, T + 2 * B,
                          n_shared=2 * B, init=init, shared_domain=max(bucket_vals + key_vals) + 1)
    m.meta.update(names=names, keys=list(keys), memos=list(memos), B=B)
    return m


def violations(m, states: np.ndarray):
    """Reachable states that break the protocol's guarantees:
    - a key stored (done, with its data) in two buckets;
    - a terminal state where some key was answered NEW by no thread or by two;
    - a thread ending FULL although the line has room for every distinct key."""
    names, keys, B = m.meta["names"], m.meta["keys"], m.meta["B"]
    T = len(keys)
    bad = []
    terminal = {names.index((NEW, -1)): NEW, names.index((SEEN, -1)): SEEN,
                names.index((FULL, -1)): FULL}
    for s in states:
        loc, b, d = s[:T], s[T:T + B], s[T + B:T + 2 * B]
        stored = [int(d[i]) for i in range(B) if b[i] > 0 and b[i] % 2 == 0]
        if len(stored) != len(set(stored)):
            bad.append(("duplicate", s.tolist()))
        if all(int(x) in terminal for x in loc):
            outcome = [terminal[int(x)] for x in loc]
            for k in set(keys):
                news = sum(1 for t in range(T) if keys[t] == k and outcome[t] == NEW)
                if news != 1 and not any(o == FULL for o in outcome):
                    bad.append(("new-count", k, s.tolist()))
            if FULL in outcome and len(set(keys)) <= B:
                bad.append(("full", s.tolist()))
    return bad
