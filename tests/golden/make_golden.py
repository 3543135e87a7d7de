"""Write the stored expected values of the large reachability cases.

Calls only the CPU oracle (oracle/) on models from the seeded generator; no
value here comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1004_2772_gb300 import synth  # noqa: E402

CASES = {
    # 12 guarded processes, 4 shared variables, mutex; 5.5M states
    "beem_medium": dict(model=dict(seed=7, update_pct=40), log2_buckets=24),
    # the BEEM-shaped workload: 12 processes, 4 shared variables in [0,4), W = 16; 32M states
    "beem_c2": dict(model=dict(seed=22, update_pct=40), log2_buckets=26),
}


def make(name):
    spec = CASES[name]
    m = synth.beem_shaped_model(**spec["model"])
    t = time.time()
    r = oracle.reach(m)
    dt = time.time() - t
    assert not r.truncated
    out = dict(spec)
    out.update(name=name, model_name=m.name, states=r.states, transitions=r.transitions,
               deadlocks=r.deadlocks, digest=f"{r.digest:#018x}", level_sizes=r.level_sizes,
               oracle_seconds=round(dt, 1),
               _about="Expected values written by tests/golden/make_golden.py from the CPU oracle "
                      "(single-threaded std::unordered_set BFS).")
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, r.states, r.transitions, len(r.level_sizes), f"{dt:.1f}s")


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["beem_medium"]):
        make(n)
