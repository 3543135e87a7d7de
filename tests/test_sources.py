"""Static checks of the CUDA sources (no GPU).

A warp-synchronous intrinsic with a full mask must be executed by every lane
the mask names.  Behind a short-circuit (`a && __shfl_sync(...)`) or in one
arm of a conditional expression it is skipped by the lanes for which the
left side already decides the result, and the warp then waits for lanes that
never arrive, or gets undefined values back.  This test keeps that form out
of the kernels.
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1004_2772_gb300", "csrc")
SYNC = r"__(shfl|shfl_up|shfl_down|shfl_xor|ballot|any|all|match_any|match_all|syncwarp|reduce_\w+)_sync\b|__syncwarp\b"
SHORT = re.compile(r"(&&|\|\||\?)\s*(" + SYNC + ")")


def _code_lines(path):
    with open(path) as f:
        for n, line in enumerate(f, 1):
            code = line.split("//", 1)[0]
            if code.strip():
                yield n, code


def test_no_warp_intrinsic_behind_a_short_circuit():
    bad = []
    for path in sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))):
        for n, code in _code_lines(path):
            if SHORT.search(code):
                bad.append(f"{os.path.basename(path)}:{n}: {code.strip()}")
    assert not bad, "warp intrinsic behind &&, || or ?:\n" + "\n".join(bad)


def test_the_check_catches_the_form():
    assert SHORT.search("const bool both = eq && __shfl_xor_sync(0xffffffffu, eq, 1);")
    assert SHORT.search("x = c ? __ballot_sync(m, p) : 0;")
    assert not SHORT.search("const bool other = __shfl_xor_sync(0xffffffffu, eq, 1) != 0;")
