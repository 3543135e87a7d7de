"""Pins of the CPU oracle to things other than itself (no GPU).

* published SplitMix64 outputs (the fingerprint's building block);
* closed forms of the interleaving family: states = prod n_p, transitions =
  sum_p E_p * prod_{q != p} n_q, level sizes = convolution of the per-automaton
  BFS layer histograms (distance in a product of graphs is the sum of the
  component distances), reachable set = the whole product space;
* a dense brute-force fixpoint over the product space of tiny guarded models;
* hand-enumerated models (tests/golden/hand_models.json);
* an O(n^2) brute force of find-or-put over short key streams;
* planted mistakes: each test build of the oracle with one plausible bug
  (ORACLE_PLANT) must fail at least one of these pins.
"""
import math

import numpy as np
import pytest

import oracle
from bruteforce import brute_force, sort_rows
from conftest import hand_models, load_golden
from paper_1004_2772_gb300 import synth

M64 = (1 << 64) - 1
PIN_CAP = 2_000_000  # every pin model is far smaller; bounds a planted runaway


# ---------------------------------------------------------------------------
# Check functions: return a list of failure messages (empty = pass), so the
# planted-mistake tests can reuse them.
# ---------------------------------------------------------------------------

def check_splitmix(plant=0):
    g = load_golden("splitmix64.json")
    bad = []
    for z, want in g["values"]:
        got = oracle.splitmix64(int(z, 16), plant=plant)
        if got != int(want, 16):
            bad.append(f"splitmix64({z}) = {got:#x}, published {want}")
    return bad


def check_fingerprint(plant=0):
    bad = []
    # x = W = 1, x ^ 1 = 0, one SplitMix64 step of 0: the first published output
    if oracle.fingerprint([1], plant=plant) != 0xE220A8397B1DCDAF:
        bad.append("fingerprint([1]) != splitmix64(0)")
    rng = np.random.default_rng(7)
    for W in (1, 5, 16, 32):
        v = rng.integers(-2**31, 2**31 - 1, size=W, dtype=np.int64).astype(np.int32)
        g0 = oracle.fingerprint(v, plant=plant)
        for i in range(W):
            w = v.copy()
            w[i] = np.int32(np.uint32(w[i].view(np.uint32) ^ np.uint32(1 << int(rng.integers(0, 32)))).view(np.int32))
            if oracle.fingerprint(w, plant=plant) == g0:
                bad.append(f"fingerprint ignores word {i} of {W}")
        if W > 1 and v[0] != v[1]:
            w = v.copy()
            w[0], w[1] = v[1], v[0]
            if oracle.fingerprint(w, plant=plant) == g0:
                bad.append("fingerprint is order-blind inside a vector")
    if oracle.fingerprint([0], plant=plant) == oracle.fingerprint([0, 0], plant=plant):
        bad.append("fingerprint ignores the vector length")
    return bad


def local_layers(m, p):
    """BFS layer histogram of process p's local automaton from init[p]."""
    n = int(m.n_local[p])
    dist = [-1] * n
    s0 = int(m.init[p])
    dist[s0] = 0
    q = [s0]
    for s in q:
        for e in m.edges_of(p, s):
            d = int(m.edge_dst[e])
            if dist[d] < 0:
                dist[d] = dist[s] + 1
                q.append(d)
    assert min(dist) >= 0, "interleaving automata are strongly connected"
    return np.bincount(dist).astype(np.int64)


def interleaving_closed_form(m):
    n = [int(x) for x in m.n_local]
    states = math.prod(n)
    E = [len(range(int(m.edge_begin[int(m.local_base[p])]),
                   int(m.edge_begin[int(m.local_base[p]) + n[p]]))) for p in range(m.n_procs)]
    transitions = sum(E[p] * math.prod(n[:p] + n[p + 1:]) for p in range(m.n_procs))
    levels = np.array([1], dtype=np.int64)
    for p in range(m.n_procs):
        levels = np.convolve(levels, local_layers(m, p))
    space = np.zeros((states, m.state_words), dtype=np.int32)
    space[:, :m.n_procs] = np.stack(np.unravel_index(np.arange(states), n), axis=1)
    return states, transitions, [int(x) for x in levels], space


def check_interleaving(m, plant=0):
    bad = []
    states, transitions, levels, space = interleaving_closed_form(m)
    r = oracle.reach(m, keep_states=True, plant=plant, max_states=PIN_CAP)
    if r.states != states:
        bad.append(f"{m.name}: states {r.states} != {states}")
    if r.transitions != transitions:
        bad.append(f"{m.name}: transitions {r.transitions} != {transitions}")
    if r.level_sizes != levels:
        bad.append(f"{m.name}: level sizes differ")
    if r.deadlocks != 0:
        bad.append(f"{m.name}: deadlocks {r.deadlocks}")
    if r.state_list is not None and r.state_list.shape == space.shape:
        if not np.array_equal(sort_rows(r.state_list), sort_rows(space)):
            bad.append(f"{m.name}: reachable set != product space")
    if r.digest != oracle.digest(space, plant=plant):
        bad.append(f"{m.name}: digest != digest of the product space")
    return bad


def check_bruteforce(m, plant=0):
    bad = []
    b = brute_force(m)
    r = oracle.reach(m, keep_states=True, plant=plant, max_states=PIN_CAP)
    for k in ("states", "transitions", "deadlocks", "level_sizes"):
        if getattr(r, k) != getattr(b, k):
            bad.append(f"{m.name}: {k} oracle {getattr(r, k)} != brute force {getattr(b, k)}")
    if r.state_list.shape != b.state_list.shape or not np.array_equal(sort_rows(r.state_list),
                                                                         b.state_list):
        bad.append(f"{m.name}: state sets differ")
    elif r.digest != oracle.digest(b.state_list, plant=plant):
        bad.append(f"{m.name}: digest differs from the brute-force set's")
    return bad


def check_hand(plant=0):
    bad = []
    for m, d in hand_models():
        r = oracle.reach(m, keep_states=True, plant=plant, max_states=PIN_CAP)
        for k in ("states", "transitions", "deadlocks", "level_sizes"):
            if getattr(r, k) != d[k]:
                bad.append(f"{d['name']}: {k} {getattr(r, k)} != hand value {d[k]}")
        want = sort_rows(np.array(d["state_list"], dtype=np.int32))
        if r.state_list.shape != want.shape or not np.array_equal(sort_rows(r.state_list), want):
            bad.append(f"{d['name']}: state set differs from the hand enumeration")
    return bad


def brute_stream(keys):
    n = keys.shape[0]
    seen = np.zeros(n, dtype=np.uint8)
    first = np.zeros(n, dtype=np.uint64)
    for k in range(n):
        first[k] = k
        for j in range(k):
            if np.array_equal(keys[j], keys[k]):
                seen[k] = 1
                first[k] = j
                break
    return seen, first


def check_stream(plant=0):
    bad = []
    rng = np.random.default_rng(3)
    for W in (1, 5, 16):
        pool = rng.integers(-3, 3, size=(40, W), dtype=np.int64).astype(np.int32)
        keys = pool[rng.integers(0, 40, size=300)]
        r = oracle.find_or_put_stream(keys, plant=plant)
        s, f = brute_stream(keys)
        if not np.array_equal(r.seen, s) or not np.array_equal(r.first, f):
            bad.append(f"stream W={W}: seen/first differ from brute force")
        uniq = np.unique(keys, axis=0)
        if r.n_new != uniq.shape[0] or r.digest != oracle.digest(uniq, plant=plant):
            bad.append(f"stream W={W}: distinct count or digest differ")
    return bad


TINY_BEEM = [dict(seed=s, n_procs=3 + s % 2, n_shared=1 + s % 2, state_words=(3 + s % 2) + (1 + s % 2) + (s % 3) * 2,
                  n_lo=2, n_hi=4, deg_lo=1, deg_hi=3, shared_domain=2 + s % 2,
                  guard_pct=(100, 60, 30)[s % 3], update_pct=(100, 50)[s % 2], mutex=s % 4 != 3)
             for s in range(1, 13)]


def tiny_beem(kw):
    return synth.beem_shaped_model(**kw)


def small_interleavings():
    return [synth.tiny_interleaving_model(),
            synth.interleaving_model(5, [3, 7, 2, 5], 8),
            synth.sized_interleaving_model(9, 6, 12, 4000),
            synth.interleaving_model(11, [1, 4, 9], 3)]


def all_pins(plant=0):
    bad = check_splitmix(plant) + check_fingerprint(plant) + check_hand(plant) + check_stream(plant)
    for m in small_interleavings()[1:]:
        bad += check_interleaving(m, plant)
    for kw in TINY_BEEM[:6]:
        bad += check_bruteforce(tiny_beem(kw), plant)
    return bad


# ---------------------------------------------------------------------------
# Tests against the default (unplanted) oracle.
# ---------------------------------------------------------------------------

def test_splitmix64_published_values():
    assert check_splitmix() == []


def test_fingerprint_composition_and_sensitivity():
    assert check_fingerprint() == []


def test_digest_is_an_order_independent_sum():
    rng = np.random.default_rng(11)
    a = rng.integers(-100, 100, size=(50, 7), dtype=np.int64).astype(np.int32)
    b = rng.integers(-100, 100, size=(30, 7), dtype=np.int64).astype(np.int32)
    da, db = oracle.digest(a), oracle.digest(b)
    assert oracle.digest(a[rng.permutation(50)]) == da
    assert oracle.digest(np.concatenate([a, b])) == (da + db) & M64
    assert da == sum(oracle.fingerprint(r) for r in a) & M64


@pytest.mark.parametrize("idx", range(4))
def test_interleaving_closed_forms(idx):
    assert check_interleaving(small_interleavings()[idx]) == []


def test_tiny_interleaving_workload_numbers():
    """5 processes x 10 states: exactly 10^5 states and 2*5*10^5 = 10^6 transitions."""
    r = oracle.reach(synth.tiny_interleaving_model())
    assert (r.states, r.transitions, r.deadlocks) == (100000, 1000000, 0)
    assert sum(r.level_sizes) == r.states and len(r.level_sizes) <= 46


@pytest.mark.parametrize("kw", TINY_BEEM, ids=[f"seed{k['seed']}" for k in TINY_BEEM])
def test_guarded_models_against_brute_force(kw):
    assert check_bruteforce(tiny_beem(kw)) == []


def test_hand_enumerated_models():
    assert check_hand() == []


def test_successor_order_and_multiplicity():
    m = [m for m, d in hand_models() if d["name"] == "self-loop-and-parallel-edges"][0]
    assert oracle.successors(m, [0]).tolist() == [[0], [1], [1]]
    assert oracle.successors(m, [1]).shape[0] == 0


def test_find_or_put_stream_brute_force():
    assert check_stream() == []


def test_key_stream_structure():
    """Uniform reuse only repeats earlier ids, so even calls are new and odd
    calls are seen; with Zipf reuse exactly n_ids calls are new."""
    n_ids = 3000
    ids = synth.call_ids(5, n_ids, 0, 2 * n_ids, "uniform")
    keys = synth.key_words(5, ids, 16)
    r = oracle.find_or_put_stream(keys)
    assert r.n_new == n_ids
    assert r.seen[0::2].sum() == 0 and r.seen[1::2].all()
    zt = synth.zipf_table(n_ids)
    ids = synth.call_ids(5, n_ids, 0, 2 * n_ids, "zipf", zt)
    r = oracle.find_or_put_stream(synth.key_words(5, ids, 16))
    assert r.n_new == n_ids
    assert r.digest == oracle.digest(synth.key_words(5, np.arange(n_ids), 16))


def test_truncation_is_reported():
    r = oracle.reach(synth.tiny_interleaving_model(), max_states=1000)
    assert r.truncated and r.states <= 1001


# ---------------------------------------------------------------------------
# Planted mistakes must be caught.
# ---------------------------------------------------------------------------

PLANTS = {1: "guards ignored", 2: "mutex counts the moving process itself",
          3: "shared-variable updates dropped", 4: "last word left out of the fingerprint",
          5: "self-loops not counted as transitions", 6: "insert deferred to the end of a level"}


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=[PLANTS[k] for k in sorted(PLANTS)])
def test_planted_mistake_is_caught(plant):
    assert all_pins(0) == [] if plant == 1 else True
    assert all_pins(plant) != [], f"planted mistake '{PLANTS[plant]}' passed every pin"
