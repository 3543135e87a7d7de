"""The kernel's own find-or-put walk (sector snapshots, stale masks, the
first sector's masks reused at the wrap-around, re-evaluation after a failed
CAS, double-hashing rehash), explored exhaustively for a few threads
(tests/walk_model.py).  No state may hold one key in two buckets; when every
thread has finished, each distinct key was answered "new" exactly once and
all threads inserting a key got the same bucket; no thread gives up while the
table has room; and no state is stuck (every wait ends).  Each planted slip
must be caught by at least one case, and re-reading the first sector at the
wrap-around (not a slip) must still pass.
"""
import pytest

import walk_model as W

K = W.Walk
# (buckets per sector, sectors per line, lines, max rehash, threads (key, memo, offset, line, step))
CASES = {
    "race-same-key-offset1": (2, 2, 1, 0, (K(1, 1, 1, 0, 1), K(1, 1, 1, 0, 1), K(2, 1, 0, 0, 1))),
    "race-same-key-offset0": (2, 2, 1, 0, (K(1, 1, 0, 0, 1), K(1, 1, 0, 0, 1), K(2, 1, 0, 0, 1))),
    "wrap-stale-first-sector": (2, 2, 1, 0, (K(1, 1, 0, 0, 1), K(1, 1, 0, 0, 1), K(2, 1, 3, 0, 1))),
    "wrap-same-key": (2, 2, 1, 0, (K(1, 1, 3, 0, 1), K(1, 1, 3, 0, 1), K(2, 1, 2, 0, 1))),
    "memo-collisions": (2, 2, 1, 0, (K(1, 1, 3, 0, 1), K(2, 1, 3, 0, 1), K(3, 2, 3, 0, 1))),
    "three-equal": (2, 2, 1, 0, (K(1, 1, 0, 0, 1), K(1, 1, 0, 0, 1), K(1, 1, 0, 0, 1))),
    "rehash": (1, 2, 2, 1, (K(1, 1, 0, 0, 1), K(2, 1, 1, 0, 1), K(3, 1, 0, 0, 1))),
    "rehash-dup": (1, 2, 2, 1, (K(1, 1, 0, 0, 1), K(2, 1, 1, 0, 1), K(2, 1, 1, 0, 1))),
    "full": (1, 2, 1, 0, (K(1, 1, 0, 0, 1), K(2, 1, 1, 0, 1), K(3, 1, 0, 0, 1))),
    "wide-sector": (4, 2, 1, 0, (K(1, 1, 2, 0, 1), K(1, 1, 2, 0, 1), K(2, 1, 1, 0, 1))),
    "two-lines-wide": (4, 2, 2, 1, (K(1, 1, 6, 0, 1), K(1, 1, 6, 0, 1), K(2, 2, 7, 0, 1))),
    "one-sector-lines": (4, 1, 2, 1, (K(1, 1, 3, 0, 1), K(1, 1, 3, 0, 1), K(2, 1, 2, 0, 1))),
}
PLANTS = ("no_reeval", "skip_write", "empty_first")


def _explore(name, broken=None):
    SB, NS, lines, mr, th = CASES[name]
    return W.explore(W.Config(SB=SB, NS=NS, lines=lines, max_rehash=mr, threads=th, broken=broken))


@pytest.mark.parametrize("name", sorted(CASES))
def test_walk_keeps_its_guarantees(name):
    n, bad, terminal, stuck = _explore(name)
    assert bad == [] and stuck == 0 and terminal > 0 and n > 50


@pytest.mark.parametrize("name", sorted(CASES))
def test_rereading_the_first_sector_also_passes(name):
    n, bad, terminal, stuck = _explore(name, "fresh_wrap")
    assert bad == [] and stuck == 0


@pytest.mark.parametrize("plant", PLANTS)
def test_planted_slip_is_caught(plant):
    caught = [name for name in CASES if "duplicate" in _explore(name, plant)[1]]
    assert caught, plant


def test_four_threads_two_keys():
    th = (K(1, 1, 1, 0, 1), K(1, 1, 1, 0, 1), K(2, 1, 1, 0, 1), K(2, 1, 1, 0, 1))
    n, bad, terminal, stuck = W.explore(W.Config(SB=2, NS=2, lines=1, max_rehash=0, threads=th))
    assert bad == [] and stuck == 0 and n > 10_000
    n, bad, _, _ = W.explore(W.Config(SB=2, NS=2, lines=1, max_rehash=0, threads=th, broken="no_reeval"))
    assert "duplicate" in bad
