"""Dense brute-force reachability over the whole product space (test helper).

Independent of the oracle's BFS and of any hashing: every state of the product
space  prod(n_local) x shared_domain^S  gets a mixed-radix index, the enabled
transitions of ALL states are computed with vectorised numpy, and reachability
is a fixpoint of frontier bitsets.  Only for tiny models (the product space is
materialised).

Model semantics (the seeded model encoding): edge e of process p leaving local
state s is enabled in v when v[p] == s, (guard_var[e] < 0 or
v[P + guard_var[e]] == guard_val[e]) and not (crit[p] >= 0 and
dst == crit[p] and some q != p has v[q] == crit[q] >= 0); firing sets v[p] = dst
and v[P + upd_var[e]] = upd_val[e] when upd_var[e] >= 0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Brute:
    states: int
    transitions: int
    deadlocks: int
    level_sizes: list
    state_list: np.ndarray  # reachable states, W words each, sorted lexicographically


def brute_force(m, max_space: int = 1 << 22) -> Brute:
    P, S, W = m.n_procs, m.n_shared, m.state_words
    D = int(m.shared_domain)
    radix = [int(x) for x in m.n_local] + [D] * S
    N = int(np.prod(radix, dtype=np.int64))
    assert N <= max_space, "product space too large for brute force"
    # comps[i, j] = component j of state i (mixed radix, component 0 most significant)
    comps = np.stack(np.unravel_index(np.arange(N), radix), axis=1).astype(np.int64)
    weights = np.array([int(np.prod(radix[j + 1:], dtype=np.int64)) for j in range(len(radix))],
                       dtype=np.int64)

    crit = np.asarray(m.crit, dtype=np.int64)
    in_crit = np.zeros((N, P), dtype=bool)
    for q in range(P):
        if crit[q] >= 0:
            in_crit[:, q] = comps[:, q] == crit[q]
    n_in_crit = in_crit.sum(axis=1)

    src_all, dst_all = [], []
    base = m.local_base
    for p in range(P):
        for s in range(int(m.n_local[p])):
            b = int(base[p]) + s
            for e in range(int(m.edge_begin[b]), int(m.edge_begin[b + 1])):
                ok = comps[:, p] == s
                gv, gc = int(m.guard_var[e]), int(m.guard_val[e])
                if gv >= 0:
                    ok &= comps[:, P + gv] == gc
                d = int(m.edge_dst[e])
                if crit[p] >= 0 and d == crit[p]:
                    others = n_in_crit - in_crit[:, p].astype(np.int64)
                    ok &= others == 0
                src = np.nonzero(ok)[0]
                tgt = comps[src].copy()
                tgt[:, p] = d
                uv, uc = int(m.upd_var[e]), int(m.upd_val[e])
                if uv >= 0:
                    tgt[:, P + uv] = uc
                src_all.append(src)
                dst_all.append(tgt @ weights)
    src = np.concatenate(src_all) if src_all else np.zeros(0, np.int64)
    dst = np.concatenate(dst_all) if dst_all else np.zeros(0, np.int64)
    outdeg = np.bincount(src, minlength=N)

    init = np.asarray(m.init[:P + S], dtype=np.int64)
    i0 = int(init @ weights)
    seen = np.zeros(N, dtype=bool)
    seen[i0] = True
    frontier = np.zeros(N, dtype=bool)
    frontier[i0] = True
    levels = [1]
    while True:
        nxt = np.zeros(N, dtype=bool)
        sel = frontier[src]
        nxt[dst[sel]] = True
        nxt &= ~seen
        k = int(nxt.sum())
        if k == 0:
            break
        levels.append(k)
        seen |= nxt
        frontier = nxt
    reach_idx = np.nonzero(seen)[0]
    transitions = int(outdeg[reach_idx].sum())
    deadlocks = int((outdeg[reach_idx] == 0).sum())
    st = np.zeros((reach_idx.shape[0], W), dtype=np.int32)
    st[:, :P + S] = comps[reach_idx]
    order = np.lexsort(st.T[::-1])
    return Brute(states=int(reach_idx.shape[0]), transitions=transitions, deadlocks=deadlocks,
                 level_sizes=levels, state_list=st[order])


def sort_rows(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a)
    return a[np.lexsort(a.T[::-1])]
