"""The stored expected values of the batched and served configurations (no GPU).

tests/golden/make_golden.py wrote them from the closed forms of the
interleaving family and the CPU oracle.  Here they are checked once more
against things other than the script: the generator still produces the same
models (names and local state counts), the counts follow from the local state
counts (states = prod n_p; transitions = 2 * states * P, since every local
state of this family has exactly two out-edges), the level sizes sum to the
states, and the smaller members equal the oracle's BFS run here.
"""
import math

import pytest

import oracle
from conftest import load_golden
from paper_1004_2772_gb300 import synth

SMALL = 60_000


def _check(models, entries):
    assert [m.name for m in models] == [e["name"] for e in entries]
    checked = 0
    for m, e in zip(models, entries):
        assert [int(x) for x in m.n_local] == e["n_local"] and m.state_words == e["state_words"]
        states = math.prod(e["n_local"])
        assert e["states"] == states
        assert e["transitions"] == 2 * states * m.n_procs
        assert e["deadlocks"] == 0 and sum(e["level_sizes"]) == states and e["level_sizes"][0] == 1
        if states <= SMALL:
            r = oracle.reach(m)
            assert (r.states, r.transitions, r.deadlocks, r.digest, r.level_sizes) == (
                e["states"], e["transitions"], e["deadlocks"], int(e["digest"], 16), e["level_sizes"])
            checked += 1
    return checked


def test_batched_golden():
    g = load_golden("batched_256.json")
    assert len(g["models"]) == 256
    assert _check(synth.batched_models(count=256, first_seed=1), g["models"]) >= 20


def test_served_golden():
    g = load_golden("served_seed5.json")
    jobs = synth.served_jobs(seed=5, rate=20.0, duration_s=10.0)
    assert len(g["jobs"]) == len(jobs) >= 150
    assert max(e["states"] for e in g["jobs"]) > 10 ** 8  # the stream reaches its largest sizes
    assert [round(a, 9) for a, _ in jobs] == [round(e["arrival_s"], 9) for e in g["jobs"]]
    assert _check([m for _, m in jobs], g["jobs"]) >= 10
