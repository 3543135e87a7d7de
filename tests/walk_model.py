"""The find-or-put walk as the CUDA table runs it, as an explicit-state model
(test helper).

tests/protocol_model.py models the protocol of Alg. "find-or-put" bucket by
bucket.  The kernel (csrc/table.cuh, find_or_put) does not act on one bucket
at a time: it reads a whole 32-byte sector of buckets, turns it into three bit
masks (empty, memo-equal, done) and then acts on those masks, which may be
stale by the time it acts.  This module models exactly that walk, so that an
exhaustive exploration of all interleavings of a few threads checks the
kernel's own reading of the paper (a stale non-empty mask bit stays true
because a used bucket never changes; a stale empty bit is corrected by the
CAS, Fig. "State diagram of buckets"):

* a line of L buckets is NS sectors of SB buckets; a key's walk starts at
  position `off` of its line: sector s0 = off // SB from position p0 =
  off % SB, then sectors s0+1, ... (cyclically), then the positions of s0
  before p0 -- for which the masks read at the first visit are reused;
* a sector is read word by word (one model step per bucket word, so reads
  interleave with every other thread's steps; an atomic 32-byte snapshot is
  one of these interleavings) and turned into the three masks;
* the first candidate in walk order that is empty or memo-equal is acted on:
  empty -> CAS(0 -> <memo, write>); success -> write the data, publish
  <memo, done>, answer NEW; failure -> the bucket is re-evaluated with the
  value the CAS returned (memo-equal -> the match path, else the walk goes on);
  memo-equal -> wait (poll, one step each) while the write bit is set, then
  compare the data: equal -> SEEN, else the walk goes on;
* after the line, the next line = (line + step) mod lines (double hashing),
  at most max_rehash further lines, then FULL.

Each thread inserts one key (key, memo, off, line0, step); threads inserting
the same key have the same hash, so the same memo, offset, line and step.

Planted mistakes (`broken`), each a plausible slip in that walk:
  "no_reeval"    a failed CAS skips the bucket instead of re-evaluating it
  "skip_write"   a memo-equal bucket still being written is skipped, not waited on
  "empty_first"  an empty bucket is taken before an earlier memo-equal one
  "fresh_wrap"   (not a mistake) the wrap-around re-reads sector s0 instead of
                 reusing its first masks -- must still pass

The steps are explored under sequential consistency: the ordering the kernel
relies on between a data row and its bucket word (gpu-scope fence before the
publish, acquire loads or fences before a row compare, Sec. 3.3) is what makes
each model step a single ordered event.
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass

# thread phases
RD, CAS, WR, PUB, POLL, CMP, NEW, SEEN, FULL = range(9)
TERMINAL = (NEW, SEEN, FULL)


@dataclass(frozen=True)
class Walk:
    key: int
    memo: int
    off: int
    line0: int
    step: int


@dataclass
class Config:
    SB: int            # buckets per sector
    NS: int            # sectors per line
    lines: int
    max_rehash: int
    threads: tuple     # Walk per thread
    broken: str | None = None

    @property
    def L(self):
        return self.SB * self.NS


# A thread's local state (a tuple, hashable):
#   (phase, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, answer_idx)
# v: visit number inside the line (0..NS); k: next word of the sector being read
# (RD); emp/mem/dn: masks of the visited sector (partial while reading);
# f*: masks of sector s0 from visit 0; todo: positions of this visit still to
# settle; pos: the position acted on; answer_idx: bucket of the answer.


def _sector_of(cfg, w, v):
    s0 = w.off // cfg.SB
    return (s0 + v) % cfg.NS


def _todo(cfg, w, v):
    p0 = w.off % cfg.SB
    full = (1 << cfg.SB) - 1
    if v == 0:
        return (full << p0) & full
    if v == cfg.NS:
        return (1 << p0) - 1
    return full


def _bucket(cfg, line, sec, pos):
    return line * cfg.L + sec * cfg.SB + pos


def _start_visit(cfg, w, st):
    """Begin visit v of the current line: read the sector, or (wrap-around)
    reuse the first visit's masks; lines exhausted -> rehash or FULL."""
    phase, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, ans = st
    while True:
        if v > cfg.NS or (v == cfg.NS and _todo(cfg, w, v) == 0):
            # line done: next line (double hashing) or give up
            if r + 1 > cfg.max_rehash:
                return (FULL, r, line, v, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1)
            r += 1
            line = (line + w.step) % cfg.lines
            v = 0
            continue
        if v == cfg.NS and cfg.broken != "fresh_wrap":
            st = (RD, r, line, v, femp, fmem, fdn, femp, fmem, fdn, _todo(cfg, w, v), 0, cfg.SB, -1)
            return _scan(cfg, w, st)
        return (RD, r, line, v, 0, 0, 0, femp, fmem, fdn, _todo(cfg, w, v), 0, 0, -1)


def _scan(cfg, w, st):
    """Masks complete: pick the first candidate of the visit, or go on."""
    phase, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, ans = st
    cand = (emp | mem) & todo
    if cfg.broken == "empty_first" and emp & todo:
        cand = emp & todo
    if not cand:
        return _start_visit(cfg, w, (RD, r, line, v + 1, 0, 0, 0, femp, fmem, fdn, 0, 0, 0, -1))
    p = (cand & -cand).bit_length() - 1
    bit = 1 << p
    base = (phase, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, p, k, -1)
    if emp & bit:
        return (CAS,) + base[1:]
    return _match(cfg, w, base)


def _match(cfg, w, st):
    """Act on memo-equal position st.pos: wait while write, else compare."""
    phase, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, ans = st
    bit = 1 << pos
    if not (dn & bit):
        if cfg.broken == "skip_write":
            return _settle(cfg, w, st)
        return (POLL,) + st[1:]
    return (CMP,) + st[1:]


def _settle(cfg, w, st):
    """Position st.pos is settled without an answer: continue the walk."""
    phase, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, ans = st
    todo &= ~((2 << pos) - 1)
    return _scan(cfg, w, (RD, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, cfg.SB, -1))


def initial(cfg):
    B = cfg.L * cfg.lines
    locs = []
    for w in cfg.threads:
        st = (RD, 0, w.line0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, -1)
        locs.append(_start_visit(cfg, w, st))
    # buckets: 0 empty, 2m-1 write(memo m), 2m done(memo m); data: key or 0;
    # ghost: key of the thread that claimed the bucket (0 = none)
    return (tuple([0] * B), tuple([0] * B), tuple([0] * B), tuple(locs))


def steps(cfg, g):
    """Successor global states: every non-terminal thread takes its next step."""
    buckets, data, ghost, locs = g
    out = []
    for t, (w, st) in enumerate(zip(cfg.threads, locs)):
        phase = st[0]
        if phase in TERMINAL:
            continue
        _, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, ans = st
        sec = _sector_of(cfg, w, v)
        nb, nd, ng = buckets, data, ghost
        if phase == RD:  # read bucket word k of the sector
            i = _bucket(cfg, line, sec, k)
            x = buckets[i]
            bit = 1 << k
            emp |= bit if x == 0 else 0
            mem |= bit if x and (x + 1) // 2 == w.memo else 0
            dn |= bit if x and x % 2 == 0 else 0
            if k + 1 == cfg.SB and v == 0:
                femp, fmem, fdn = emp, mem, dn  # the first sector as read, kept for the wrap-around
            ns = (RD, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k + 1, -1)
            if k + 1 == cfg.SB:
                ns = _scan(cfg, w, ns)
        elif phase == CAS:
            i = _bucket(cfg, line, sec, pos)
            old = buckets[i]
            if old == 0:
                nb = buckets[:i] + (2 * w.memo - 1,) + buckets[i + 1:]
                ng = ghost[:i] + (w.key,) + ghost[i + 1:]
                ns = (WR,) + st[1:13] + (i,)
            else:
                bit = 1 << pos
                emp &= ~bit
                if cfg.broken == "no_reeval":
                    ns = _settle(cfg, w, (RD, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, -1))
                else:
                    mem = (mem | bit) if (old + 1) // 2 == w.memo else (mem & ~bit)
                    dn = (dn | bit) if old % 2 == 0 else (dn & ~bit)
                    st2 = (RD, r, line, v, emp, mem, dn, femp, fmem, fdn, todo, pos, k, -1)
                    ns = _match(cfg, w, st2) if mem & bit else _settle(cfg, w, st2)
        elif phase == WR:
            nd = data[:ans] + (w.key,) + data[ans + 1:]
            ns = (PUB,) + st[1:]
        elif phase == PUB:
            nb = buckets[:ans] + (2 * w.memo,) + buckets[ans + 1:]
            ns = (NEW,) + st[1:]
        elif phase == POLL:
            i = _bucket(cfg, line, sec, pos)
            if buckets[i] % 2 == 0:  # done
                ns = (CMP,) + st[1:]
            else:
                ns = st               # still being written: poll again
        elif phase == CMP:
            i = _bucket(cfg, line, sec, pos)
            if data[i] == w.key:
                ns = (SEEN,) + st[1:13] + (i,)
            else:
                ns = _settle(cfg, w, st)
        else:
            raise AssertionError(phase)
        out.append((nb, nd, ng, locs[:t] + (ns,) + locs[t + 1:]))
    return out


def violations(cfg, g):
    """Broken guarantees in global state g:
      duplicate  two claimed buckets hold (or are being written with) one key
      new-count  all threads finished, and a key was answered NEW by no thread
                 or by two (Sec. 3.1: exactly one insert per distinct key)
      idx        two threads with the same key answered with different buckets,
                 or a SEEN answer points at a bucket not holding the key
      full       a thread gave up although the table has room for every key
    """
    buckets, data, ghost, locs = g
    bad = []
    claimed = [x for x in ghost if x]
    if len(claimed) != len(set(claimed)):
        bad.append("duplicate")
    if all(st[0] in TERMINAL for st in locs):
        keys = [w.key for w in cfg.threads]
        distinct = set(keys)
        if any(st[0] == FULL for st in locs):
            if len(distinct) <= cfg.L * cfg.lines:
                bad.append("full")
        else:
            for key in distinct:
                news = sum(1 for w, st in zip(cfg.threads, locs) if w.key == key and st[0] == NEW)
                if news != 1:
                    bad.append("new-count")
                idxs = {st[13] for w, st in zip(cfg.threads, locs) if w.key == key}
                if len(idxs) != 1 or data[next(iter(idxs))] != key:
                    bad.append("idx")
    return bad


def explore(cfg, limit: int = 3_000_000):
    """All reachable global states (BFS).  Returns (states, violations found,
    terminal states, states with no successor that are not terminal)."""
    g0 = initial(cfg)
    seen = {g0}
    queue = deque([g0])
    found, terminal, stuck = set(), 0, 0
    while queue:
        g = queue.popleft()
        for v in violations(cfg, g):
            found.add(v)
        nxt = steps(cfg, g)
        if not nxt:
            if all(st[0] in TERMINAL for st in g[3]):
                terminal += 1
            else:
                stuck += 1
        for h in nxt:
            if h not in seen:
                seen.add(h)
                if len(seen) > limit:
                    raise RuntimeError("state space larger than the limit")
                queue.append(h)
    return len(seen), sorted(found), terminal, stuck
