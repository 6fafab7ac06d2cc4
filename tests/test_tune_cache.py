"""The autotuner's cache file (host only, no GPU): choices written for some
keys are read back exactly, a later write replaces the line of the same key
and keeps the others, unknown keys and malformed lines are not found, and
keys with invalid GPU names are rejected."""
import pytest

import paper_1703_03676_gb300 as eng


def key(**kw):
    k = dict(L=64, spin_format=eng.SPIN_BITS32, dim=2, potts_q=0, r_log2=14, batched=0, sms=152,
             gpu="NVIDIA GB300")
    k.update(kw)
    return k


def test_round_trip(tmp_path):
    path = str(tmp_path / "tune.txt")
    a, b = key(), key(L=16, r_log2=9, spin_format=eng.SPIN_INT8)
    ca = {"group_threads": 32, "block_warps": 8, "attempts_per_ns": 1748.125}
    cb = {"group_threads": 32, "block_warps": 4, "attempts_per_ns": 118.0625}
    assert eng.tune_cache_lookup(path, a) is None  # no file yet
    eng.tune_cache_store(path, a, ca)
    eng.tune_cache_store(path, b, cb)
    got = eng.tune_cache_lookup(path, a)
    assert got == {**ca, "candidates": 0}
    assert eng.tune_cache_lookup(path, b) == {**cb, "candidates": 0}
    # a new choice for a replaces its line; b stays
    ca2 = {"group_threads": 16, "block_warps": 2, "attempts_per_ns": 1700.5}
    eng.tune_cache_store(path, a, ca2)
    assert eng.tune_cache_lookup(path, a) == {**ca2, "candidates": 0}
    assert eng.tune_cache_lookup(path, b) == {**cb, "candidates": 0}
    lines = open(path).read().splitlines()
    assert len(lines) == 2 and all(ln.startswith("v1|") for ln in lines)
    # every key field separates entries
    for f, v in [("L", 128), ("spin_format", eng.SPIN_MSC32), ("dim", 3), ("potts_q", 3), ("r_log2", 15),
                 ("batched", 1), ("sms", 148), ("gpu", "NVIDIA B200")]:
        assert eng.tune_cache_lookup(path, key(**{f: v})) is None, f


def test_malformed_lines_are_ignored(tmp_path):
    path = tmp_path / "tune.txt"
    path.write_text("garbage\nv1|64|1|2|0|14|0|152|NVIDIA GB300|x|8|1.0\nv2|64|1|2|0|14|0|152|NVIDIA GB300|32|8|1\n"
                    "v1|64|1|2|0|14|0|152|NVIDIA GB300|32|8\n")
    assert eng.tune_cache_lookup(str(path), key()) is None
    eng.tune_cache_store(str(path), key(), {"group_threads": 32, "block_warps": 8, "attempts_per_ns": 1.0})
    assert eng.tune_cache_lookup(str(path), key())["group_threads"] == 32
    assert len(path.read_text().splitlines()) == 1  # malformed lines dropped on rewrite


@pytest.mark.parametrize("bad", ["", "a|b", "x\ny"])
def test_bad_gpu_names_rejected(tmp_path, bad):
    with pytest.raises(eng.PAError) as ei:
        eng.tune_cache_store(str(tmp_path / "t.txt"), key(gpu=bad),
                             {"group_threads": 4, "block_warps": 8, "attempts_per_ns": 1.0})
    assert ei.value.kind == "invalid argument"
