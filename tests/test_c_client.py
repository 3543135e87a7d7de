"""The library's C ABI from a plain C program (tests/c_client/reach_client.c):
no Python binding and no torch between the caller and the entry points.

On the CPU the client must compile and link against the header and the
library (the header is valid C); on a GPU its results must equal the oracle's
for the model it builds.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1004_2772_gb300 import _build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "reach_client.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(out_dir):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = _build.build()
    libdir = os.path.dirname(lib)
    exe = os.path.join(out_dir, "reach_client")
    cuda_lib = os.path.join(CUDA, "lib64")
    cmd = [gcc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), SRC, "-o", exe, "-L", libdir, "-l:" + os.path.basename(lib),
           "-L", cuda_lib, "-lcudart", f"-Wl,-rpath,{libdir}:{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _model(P, n):
    edges = [[[((s + 1) % n, -1, 0, -1, 0), (s, -1, 0, -1, 0)] for s in range(n)] for _ in range(P)]
    return synth.build_model(f"cycle-selfloop-P{P}-n{n}", [n] * P, edges, P)


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(_compile(str(tmp_path)))


@pytest.mark.gpu
@pytest.mark.parametrize("P,n,log2", [(5, 10, 18), (3, 7, 10)])
def test_c_client_matches_oracle(cuda_lib, tmp_path, P, n, log2):
    exe = _compile(str(tmp_path))
    r = subprocess.run([exe, str(P), str(n), str(log2)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    states, transitions, deadlocks, levels, digest, seen0, seen1 = (int(x) for x in r.stdout.split())
    ref = oracle.reach(_model(P, n))
    assert (states, transitions, deadlocks, levels, digest) == (
        ref.states, ref.transitions, ref.deadlocks, len(ref.level_sizes), ref.digest)
    # closed forms of this model: n^P states, 2P successors each, P(n-1) + 1 levels
    assert states == n ** P and transitions == 2 * P * n ** P and levels == P * (n - 1) + 1
    assert (seen0, seen1) == (0, 1)
