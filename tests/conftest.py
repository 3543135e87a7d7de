import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, TESTS):
    if p not in sys.path:
        sys.path.insert(0, p)

GOLDEN = os.path.join(TESTS, "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def hand_models():
    """Models of tests/golden/hand_models.json as synth.Model objects."""
    from paper_1004_2772_gb300 import synth
    out = []
    for d in load_golden("hand_models.json")["models"]:
        m = synth.build_model(d["name"], d["n_local"], [[[tuple(e) for e in es] for es in ep]
                                                        for ep in d["edges"]],
                              d["state_words"], n_shared=d["n_shared"], crit=d["crit"],
                              shared_domain=2)
        out.append((m, d))
    return out


@pytest.fixture(scope="session")
def cuda_lib():
    """The built CUDA library (GPU tests only)."""
    import torch
    from paper_1004_2772_gb300 import _build, binding
    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    binding.load()
    return binding
