"""The autotuner: its search space (host logic, no GPU) and, on the GPU, that
every candidate of a tuning run reproduces the oracle's answer."""
import pytest

import oracle
from paper_1004_2772_gb300 import autotune, synth


def test_candidates_respect_line_lengths_per_width():
    cands = list(autotune._candidates(autotune.TABLE_SPACE))
    # one lane per key: 32-bit 3 lines x 2 dedup x 2 block sizes, 16-bit 2 x 2 x 2;
    # groups of 2, 4, 8 lanes: one line each (32-bit, no dedup) x 2 block sizes
    assert len(cands) == 12 + 8 + 3 * 2
    for c in cands:
        assert c["line_buckets"] in autotune.LINES_FOR_WIDTH[c["bucket_bits"]]
        if c["group_lanes"] > 1:
            assert c["line_buckets"] == 4 * c["group_lanes"] and c["bucket_bits"] == 32
            assert c["dedup"] == 0
    assert len({tuple(sorted(c.items())) for c in cands}) == len(cands)
    reach = list(autotune._candidates(autotune.REACH_SPACE))
    # one lane per successor: 32-bit 3 lines + 16-bit 2; groups of 2, 4, 8: one line each
    assert len(reach) == (3 + 2 + 3) * 2
    assert all(c["line_buckets"] == 4 * c["group_lanes"] for c in reach if c["group_lanes"] > 1)
    probe = list(autotune._candidates(autotune.PROBE_SPACE))
    assert len(probe) == 2 * 3 and {"rehash": 1, "max_rehash": 16} in probe


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    autotune._save_cache(path, {"k": {"best": {"line_buckets": 8}}})
    assert autotune._load_cache(path) == {"k": {"best": {"line_buckets": 8}}}
    assert autotune._load_cache(str(tmp_path / "missing.json")) == {}


@pytest.mark.gpu
def test_tune_table_candidates_agree_with_oracle(cuda_lib, tmp_path):
    n_log2, lf = 16, 0.5
    n_ids = int(lf * (1 << n_log2))
    space = {"line_buckets": (8, 16), "bucket_bits": (32, 16), "dedup": (0,), "block_threads": (256,)}
    probe = {"rehash": (0, 1), "max_rehash": (0, 64)}
    e = autotune.tune_table(n_log2, lf, "uniform", 16, seed=3, space=space, probe_space=probe, reps=1,
                            cache_path=str(tmp_path / "c.json"))
    ids = synth.call_ids(3, n_ids, 0, 2 * n_ids, "uniform")
    ref = oracle.find_or_put_stream(synth.key_words(3, ids, 16))
    assert e["n_new"] == ref.n_new == n_ids
    assert int(e["digest"], 16) == ref.digest
    # 3 layouts ((32, 8), (32, 16), (16, 16)), then 3 probe sequences on the best
    assert [r["stage"] for r in e["all"]] == ["layout"] * 3 + ["probe"] * 3
    assert all(r["admissible"] for r in e["all"])


@pytest.mark.gpu
def test_tune_table_rejects_a_bound_too_small(cuda_lib, tmp_path):
    """At load 0.97 with 8-bucket lines, one line of probing is not enough
    for every key: that candidate fails (HT_ERR_FULL) and is not chosen; the
    others agree with the oracle."""
    n_log2, lf = 14, 0.97
    n_ids = int(lf * (1 << n_log2))
    e = autotune.tune_table(n_log2, lf, "uniform", 16, seed=4,
                            space={"line_buckets": (8,), "bucket_bits": (32,), "dedup": (0,),
                                   "block_threads": (256,)},
                            probe_space={"rehash": (0, 1), "max_rehash": (0, 1)}, reps=1,
                            cache_path=str(tmp_path / "c.json"))
    ids = synth.call_ids(4, n_ids, 0, 2 * n_ids, "uniform")
    ref = oracle.find_or_put_stream(synth.key_words(4, ids, 16))
    assert (e["n_new"], int(e["digest"], 16)) == (ref.n_new, ref.digest)
    bad = [r for r in e["all"] if not r["admissible"]]
    assert bad and all(r["params"]["max_rehash"] == 1 for r in bad)
    assert e["best"].get("max_rehash", 0) != 1


@pytest.mark.gpu
def test_tune_reach_candidates_agree_with_oracle(cuda_lib, tmp_path):
    m = synth.tiny_interleaving_model()
    ref = oracle.reach(m)
    space = {"line_buckets": (8, 16), "bucket_bits": (32, 16), "block_threads": (256,)}
    e = autotune.tune_reach(m, 18, space=space, reps=1, cache_path=str(tmp_path / "c.json"))
    assert (e["states"], e["transitions"], e["deadlocks"], int(e["digest"], 16), e["level_sizes"]) == (
        ref.states, ref.transitions, ref.deadlocks, ref.digest, ref.level_sizes)
    # 3 layouts, the next-line rule on the best, then one more table doubling
    assert [r["stage"] for r in e["all"]] == ["layout"] * 3 + ["probe", "load"]
    assert e["all"][-1]["params"]["log2_buckets"] == 19 and "log2_buckets" in e["best"]
