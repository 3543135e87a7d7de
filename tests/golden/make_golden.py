"""Write the stored expected values of the large reachability cases.

Calls only the CPU oracle (oracle/) on models from the seeded generator, and,
for the interleaving family, the closed forms of tests/closed_forms.py (whose
only method arithmetic is the oracle's fingerprint); no value here comes from
the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

Cases:
  beem_medium, beem_c2   BEEM-shaped models: the oracle's BFS
  batched_256            the 256 batched models (seeds 1..256): closed forms,
                         each checked against the oracle's BFS
  served_seed5           the served Poisson stream (seed 5, 20 jobs/s, 10 s):
                         closed forms; jobs of at most 2*10^6 states are also
                         checked against the oracle's BFS
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TESTS = os.path.dirname(HERE)
ROOT = os.path.dirname(TESTS)
sys.path.insert(0, ROOT)
sys.path.insert(0, TESTS)

import oracle  # noqa: E402
from paper_1004_2772_gb300 import synth  # noqa: E402

ABOUT = ("Expected values written by tests/golden/make_golden.py from the CPU oracle "
         "(single-threaded std::unordered_set BFS)")

BEEM_CASES = {
    # 12 guarded processes, 4 shared variables, mutex; 5.5M states
    "beem_medium": dict(model=dict(seed=7, update_pct=40), log2_buckets=24),
    # the BEEM-shaped workload: 12 processes, 4 shared variables in [0,4), W = 16; 32M states
    "beem_c2": dict(model=dict(seed=22, update_pct=40), log2_buckets=26),
}
ORACLE_CHECK_STATES = 2_000_000


def make_beem(name):
    spec = BEEM_CASES[name]
    m = synth.beem_shaped_model(**spec["model"])
    t = time.time()
    r = oracle.reach(m)
    dt = time.time() - t
    assert not r.truncated
    out = dict(spec)
    out.update(name=name, model_name=m.name, states=r.states, transitions=r.transitions,
               deadlocks=r.deadlocks, digest=f"{r.digest:#018x}", level_sizes=r.level_sizes,
               oracle_seconds=round(dt, 1), _about=ABOUT + ".")
    return out


def family_entries(models, check_all):
    """Closed-form values of interleaving models, cross-checked with the
    oracle's BFS (every model, or those of at most ORACLE_CHECK_STATES)."""
    import closed_forms
    entries, checked = [], 0
    for m in models:
        e = closed_forms.expected(m)
        if check_all or e["states"] <= ORACLE_CHECK_STATES:
            r = oracle.reach(m)
            assert not r.truncated
            got = dict(states=r.states, transitions=r.transitions, deadlocks=r.deadlocks,
                       level_sizes=r.level_sizes, digest=r.digest)
            assert got == e, f"{m.name}: oracle {got} != closed form {e}"
            checked += 1
        entries.append(dict(name=m.name, state_words=m.state_words, n_local=[int(x) for x in m.n_local],
                            states=e["states"], transitions=e["transitions"], deadlocks=e["deadlocks"],
                            digest=f"{e['digest']:#018x}", level_sizes=e["level_sizes"]))
    return entries, checked


def make_batched():
    t = time.time()
    models = synth.batched_models(count=256, first_seed=1)
    entries, checked = family_entries(models, check_all=True)
    return dict(name="batched_256", generator="synth.batched_models(count=256, first_seed=1)",
                models=entries, oracle_checked=checked, seconds=round(time.time() - t, 1),
                _about=ABOUT + " and the closed forms of the interleaving family "
                       "(tests/closed_forms.py); every model's closed form equals the oracle's BFS.")


def make_served():
    t = time.time()
    jobs = synth.served_jobs(seed=5, rate=20.0, duration_s=10.0)
    entries, checked = family_entries([m for _, m in jobs], check_all=False)
    for e, (arrival, _) in zip(entries, jobs):
        e["arrival_s"] = arrival
    return dict(name="served_seed5", generator="synth.served_jobs(seed=5, rate=20.0, duration_s=10.0)",
                jobs=entries, oracle_checked=checked, seconds=round(time.time() - t, 1),
                _about=ABOUT + " and the closed forms of the interleaving family "
                       f"(tests/closed_forms.py); jobs of at most {ORACLE_CHECK_STATES} states "
                       "were checked against the oracle's BFS.")


def make(name):
    if name in BEEM_CASES:
        out = make_beem(name)
    elif name == "batched_256":
        out = make_batched()
    elif name == "served_seed5":
        out = make_served()
    else:
        raise SystemExit(f"unknown case {name}")
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=None, separators=(",", ":"))
        f.write("\n")
    print(name, "written")


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["beem_medium"]):
        make(n)
