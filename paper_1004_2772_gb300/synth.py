"""Seeded synthetic inputs: reachability models and find_or_put key streams.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from.  It draws random numbers and lays out model tables; it holds none
of the method's arithmetic (no table hash, no probing, no search, no digest).

Models follow the interleaving-automata shape of explicit-state model checking
(Section 2, Alg. "Reachability analysis"): a state vector is a fixed-length
int32 vector (Section 3.1 asks for vectors of a known length) holding

    v[0 .. P)           local state of each of the P processes
    v[P .. P+S)         S shared variables
    v[P+S .. W)         padding, always 0 (hashed, stored and compared)

The transition relation is encoded per process as a CSR edge list over its
local states.  Edge e of process p leaving local state s is enabled in v when

    v[p] == s
    and (guard_var[e] < 0 or v[P + guard_var[e]] == guard_val[e])
    and not (crit[p] >= 0 and edge_dst[e] == crit[p]
             and some q != p has crit[q] >= 0 and v[q] == crit[q])

and firing it sets v[p] = edge_dst[e] and, if upd_var[e] >= 0,
v[P + upd_var[e]] = upd_val[e].  Successors are listed for p ascending, then
edges in CSR order; every enabled edge is one transition, self-loops and
parallel edges included.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its published
definition.  uniform(a, b) = a + (x mod (b - a + 1)); the modulo bias is part of
the definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64_mix(z: int) -> int:
    """One SplitMix64 output: advance by the golden gamma, then the two
    xor-shift-multiply rounds and a final xor-shift (Steele et al. 2014)."""
    z = (z + GOLDEN_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential SplitMix64 stream: state += gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        out = splitmix64_mix(self.state)
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        return out

    def uniform(self, a: int, b: int) -> int:
        """Integer in [a, b]: a + (x mod (b - a + 1))."""
        assert b >= a
        return a + self.next() % (b - a + 1)

    def unit(self) -> float:
        """Float in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


@dataclass
class Model:
    """A model in the CSR encoding described in the module docstring."""

    name: str
    n_procs: int
    n_shared: int
    state_words: int
    n_local: np.ndarray          # int32[P]
    crit: np.ndarray             # int32[P], -1 = no critical state
    edge_begin: np.ndarray       # int32[sum(n_local) + 1]
    edge_dst: np.ndarray         # int32[E]
    guard_var: np.ndarray        # int32[E], -1 = unguarded
    guard_val: np.ndarray        # int32[E]
    upd_var: np.ndarray          # int32[E], -1 = no update
    upd_val: np.ndarray          # int32[E]
    init: np.ndarray             # int32[W]
    shared_domain: int = 4       # shared variables range over [0, shared_domain)
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.edge_dst.shape[0])

    @property
    def local_base(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_local)[:-1]]).astype(np.int64)

    def edges_of(self, p: int, s: int) -> range:
        b = int(self.local_base[p]) + s
        return range(int(self.edge_begin[b]), int(self.edge_begin[b + 1]))

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.n_local, self.crit, self.edge_begin, self.edge_dst,
                                      self.guard_var, self.guard_val, self.upd_var, self.upd_val,
                                      self.init))


def _i32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def build_model(name, n_local, edges, state_words, n_shared=0, crit=None, init=None,
                shared_domain=4, meta=None) -> Model:
    """Assemble a Model from per-(process, local state) edge lists.

    edges[p][s] is a list of (dst, guard_var, guard_val, upd_var, upd_val).
    """
    P = len(n_local)
    assert state_words >= P + n_shared, "state vector too short for processes + shared vars"
    begin = [0]
    dst, gv, gc, uv, uc = [], [], [], [], []
    for p in range(P):
        assert len(edges[p]) == n_local[p]
        for s in range(n_local[p]):
            for (d, g, c, u, c2) in edges[p][s]:
                assert 0 <= d < n_local[p]
                dst.append(d); gv.append(g); gc.append(c); uv.append(u); uc.append(c2)
            begin.append(len(dst))
    if crit is None:
        crit = [-1] * P
    if init is None:
        init = [0] * state_words
    return Model(name=name, n_procs=P, n_shared=n_shared, state_words=state_words,
                 n_local=_i32(n_local), crit=_i32(crit), edge_begin=_i32(begin),
                 edge_dst=_i32(dst), guard_var=_i32(gv), guard_val=_i32(gc),
                 upd_var=_i32(uv), upd_val=_i32(uc), init=_i32(init),
                 shared_domain=shared_domain, meta=dict(meta or {}))


# ---------------------------------------------------------------------------
# Interleaving family: independent strongly connected local automata.
# ---------------------------------------------------------------------------

def interleaving_model(seed: int, n_local, state_words: int, name: str | None = None) -> Model:
    """P independent processes; local state s has two out-edges, s -> (s+1) mod n
    (the forced cycle that makes each automaton strongly connected) and
    s -> uniform(0, n-1) (self-loops and duplicates allowed).  No shared
    variables, no guards, no critical sections; init is all zeros."""
    rng = SplitMix64(seed)
    P = len(n_local)
    edges = []
    for p in range(P):
        n = int(n_local[p])
        ep = []
        for s in range(n):
            ep.append([((s + 1) % n, -1, 0, -1, 0), (rng.uniform(0, n - 1), -1, 0, -1, 0)])
        edges.append(ep)
    return build_model(name or f"interleaving-s{seed}-P{P}-W{state_words}", list(map(int, n_local)),
                       edges, state_words, meta={"family": "interleaving", "seed": seed})


def tiny_interleaving_model() -> Model:
    """5 processes x 10 local states, 5 int32 words: 10^5 states, 10^6 transitions."""
    return interleaving_model(1, [10] * 5, 5, name="tiny-interleaving-P5-n10-W5")


def sized_interleaving_model(seed: int, n_procs: int, state_words: int, target_states: int,
                             name: str | None = None) -> Model:
    """Interleaving model whose product of local-state counts is close to
    target_states: every process gets floor(target^(1/P)) states (at least 2),
    then processes are bumped by one, lowest index first, while the product
    stays <= target."""
    assert state_words >= n_procs
    base = max(2, int(math.floor(target_states ** (1.0 / n_procs) + 1e-9)))
    n_local = [base] * n_procs
    for p in range(n_procs):
        trial = n_local.copy()
        trial[p] += 1
        if math.prod(trial) <= target_states:
            n_local = trial
    m = interleaving_model(seed, n_local, state_words,
                           name=name or f"interleaving-s{seed}-P{n_procs}-W{state_words}")
    m.meta["target_states"] = target_states
    return m


def batched_models(count: int = 256, first_seed: int = 1, lo: float = 1e3, hi: float = 1e6):
    """Models of the interleaving family with uneven sizes: for seed k,
    P = uniform(3, 12), W = uniform(max(8, P), 32), target states log-uniform
    in [lo, hi]."""
    out = []
    for k in range(first_seed, first_seed + count):
        rng = SplitMix64(0xBA7C4ED0 ^ k)
        P = rng.uniform(3, 12)
        W = rng.uniform(max(8, P), 32)
        target = int(round(10 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * rng.unit())))
        out.append(sized_interleaving_model(k, P, W, target, name=f"batched-{k}"))
    return out


# ---------------------------------------------------------------------------
# BEEM-shaped family: guarded edges over shared variables plus a mutex.
# ---------------------------------------------------------------------------

def beem_shaped_model(seed: int, n_procs: int = 12, n_shared: int = 4, state_words: int = 16,
                      n_lo: int = 4, n_hi: int = 8, deg_lo: int = 1, deg_hi: int = 3,
                      shared_domain: int = 4, guard_pct: int = 100, update_pct: int = 100,
                      mutex: bool = True, name: str | None = None) -> Model:
    """Processes with n_p = uniform(n_lo, n_hi) local states and out-degree
    uniform(deg_lo, deg_hi) per state.  Edge 0 of state s goes to (s+1) mod n_p,
    the others to uniform destinations.  Each edge, with probability
    guard_pct/100, is guarded by (shared var g == c) and, with probability
    update_pct/100, updates (shared var u := c'), g, u uniform over the shared
    variables and c, c' uniform over [0, shared_domain).  With mutex, the
    critical state of process p is n_p - 1 and at most one process may be in
    its critical state.  Draw order: all n_p; then per process, per state: the
    out-degree, then per edge: dst (edges after the first), guard coin, g, c,
    update coin, u, c'."""
    assert state_words >= n_procs + n_shared
    rng = SplitMix64(seed)
    n_local = [rng.uniform(n_lo, n_hi) for _ in range(n_procs)]
    edges = []
    for p in range(n_procs):
        n = n_local[p]
        ep = []
        for s in range(n):
            deg = rng.uniform(deg_lo, deg_hi)
            es = []
            for k in range(deg):
                d = (s + 1) % n if k == 0 else rng.uniform(0, n - 1)
                guarded = rng.uniform(0, 99) < guard_pct
                g = rng.uniform(0, n_shared - 1)
                c = rng.uniform(0, shared_domain - 1)
                upd = rng.uniform(0, 99) < update_pct
                u = rng.uniform(0, n_shared - 1)
                c2 = rng.uniform(0, shared_domain - 1)
                es.append((d, g if guarded and n_shared else -1, c if guarded and n_shared else 0,
                           u if upd and n_shared else -1, c2 if upd and n_shared else 0))
            ep.append(es)
        edges.append(ep)
    crit = [n - 1 for n in n_local] if mutex else [-1] * n_procs
    return build_model(name or f"beem-shaped-s{seed}-P{n_procs}-S{n_shared}-W{state_words}",
                       n_local, edges, state_words, n_shared=n_shared, crit=crit,
                       shared_domain=shared_domain,
                       meta={"family": "beem-shaped", "seed": seed, "guard_pct": guard_pct,
                             "update_pct": update_pct, "mutex": mutex})


# ---------------------------------------------------------------------------
# find_or_put key streams (hash-table microbenchmark).
# ---------------------------------------------------------------------------

def _mix_u64(z: np.ndarray) -> np.ndarray:
    """Vectorised SplitMix64 output function over uint64 counters."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _fmix32(x: np.ndarray) -> np.ndarray:
    """MurmurHash3 32-bit finaliser (Appleby), a bijection on uint32."""
    with np.errstate(over="ignore"):
        x = x.astype(np.uint32)
        x ^= x >> np.uint32(16)
        x *= np.uint32(0x85EBCA6B)
        x ^= x >> np.uint32(13)
        x *= np.uint32(0xC2B2AE35)
        x ^= x >> np.uint32(16)
        return x


def key_words(seed: int, ids: np.ndarray, state_words: int = 16) -> np.ndarray:
    """Key of each id: word 0 = fmix32(id) (distinct ids give distinct keys);
    words 2q-1 and 2q (q >= 1) = the low and high 32 bits of
    mix((seed << 36) + (id << 4) + q), one SplitMix64 output per two words."""
    ids = np.asarray(ids, dtype=np.uint64)
    out = np.empty((ids.shape[0], state_words), dtype=np.uint32)
    out[:, 0] = _fmix32(ids.astype(np.uint32))
    base = (np.uint64((seed << 36) & MASK64) + (ids << np.uint64(4)))
    for q in range(1, (state_words + 1) // 2 + 1):
        with np.errstate(over="ignore"):
            z = _mix_u64(base + np.uint64(q))
        for j, part in ((2 * q - 1, z & np.uint64(0xFFFFFFFF)), (2 * q, z >> np.uint64(32))):
            if j < state_words:
                out[:, j] = part.astype(np.uint32)
    return out.view(np.int32)


def mulhi_range(r: np.ndarray, n: np.ndarray) -> np.ndarray:
    """floor(r * n / 2^64) for uint64 r and 1 <= n < 2^32 (a multiply-high
    range reduction of r onto [0, n)), exactly, in 64-bit arithmetic."""
    r = np.asarray(r, dtype=np.uint64)
    n = np.asarray(n, dtype=np.uint64)
    lo32 = np.uint64(0xFFFFFFFF)
    with np.errstate(over="ignore"):
        hi = (r >> np.uint64(32)) * n
        lo = (r & lo32) * n
        return (hi + (lo >> np.uint64(32))) >> np.uint64(32)


ZIPF_CELLS = 1 << 16


def zipf_table(n_ids: int, s: float = 1.1, cells: int = ZIPF_CELLS) -> np.ndarray:
    """Quantile table of a Zipf(s) law over ranks 1..n_ids: entry k is the
    rank at cumulative probability k / cells (continuous approximation of the
    harmonic sum), entry `cells` = n_ids + 1.  A sample picks a cell from the
    top 16 bits of a random word and a rank uniformly inside the cell, so both
    sides of a parity test draw identical integers from the same table."""
    a = 1.0 - s
    total = (n_ids ** a - 1.0) / a + 1.0          # H(n) ~ 1 + int_1^n x^-s dx
    q = np.arange(cells + 1, dtype=np.float64) / cells
    target = q * total
    # invert H(r) = 1 + (r^a - 1)/a for r >= 1 (rank 1 holds the first unit of mass)
    r = np.where(target <= 1.0, 1.0, (1.0 + a * (target - 1.0)) ** (1.0 / a))
    ranks = np.clip(np.floor(r), 1, n_ids).astype(np.int64)
    ranks = np.maximum.accumulate(ranks)
    ranks[-1] = n_ids + 1
    return ranks.astype(np.uint32)


def call_ids(seed: int, n_ids: int, start: int, count: int, dist: str = "uniform",
             table: np.ndarray | None = None) -> np.ndarray:
    """Key ids of calls start .. start+count of a fill with n_ids distinct keys
    and 2 * n_ids calls.  Call 2i inserts id i; call 2i+1 repeats an id drawn
    from r = mix(mix(seed) ^ c): uniform over [0, i] ('an earlier key', as
    floor(r * (i + 1) / 2^64)), or
    Zipf over ranks 1..n_ids (id = rank - 1, id 0 hottest) through the
    quantile table.  So half the calls are duplicates and exactly n_ids keys
    are distinct."""
    c = np.arange(start, start + count, dtype=np.uint64)
    i = c >> np.uint64(1)
    odd = (c & np.uint64(1)) == np.uint64(1)
    key = np.uint64(splitmix64_mix(seed & MASK64))
    r = _mix_u64(c ^ key)
    if dist == "uniform":
        dup = mulhi_range(r, i + np.uint64(1))
    elif dist == "zipf":
        assert table is not None and table.shape[0] == ZIPF_CELLS + 1
        cell = (r >> np.uint64(48)).astype(np.int64)
        lo = table[cell].astype(np.uint64)
        hi = table[cell + 1].astype(np.uint64)
        width = np.maximum(hi - lo, np.uint64(1))
        rank = lo + (r & np.uint64(0xFFFFFFFF)) % width
        dup = np.minimum(rank, np.uint64(n_ids)) - np.uint64(1)
    else:
        raise ValueError(dist)
    return np.where(odd, dup, i).astype(np.uint64)


# ---------------------------------------------------------------------------
# Served reachability: a Poisson stream of interleaving-family jobs.
# ---------------------------------------------------------------------------

def served_jobs(seed: int = 5, rate: float = 20.0, duration_s: float = 10.0, lo: float = 1e4,
                hi: float = 2e8, state_words: int = 16, max_jobs: int | None = None):
    """[(arrival_s, model)]: exponential inter-arrival gaps of mean 1/rate,
    target sizes log-uniform in [lo, hi], P = uniform(3, 8) processes."""
    rng = SplitMix64(seed)
    t, out, k = 0.0, [], 0
    while True:
        t += -math.log(1.0 - rng.unit()) / rate
        if t > duration_s or (max_jobs is not None and len(out) >= max_jobs):
            break
        target = int(round(10 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * rng.unit())))
        P = rng.uniform(3, 8)
        k += 1
        out.append((t, sized_interleaving_model(seed * 100003 + k, P, state_words, target,
                                                name=f"served-{seed}-{k}")))
    return out
