"""The autotuner (pa_autotune): it picks a launch shape the run accepts,
remembers it in the process and in its cache file, later runs that leave
the shape open use it, and no shape changes any result: runs with the tuned
shape and with other shapes give the same rows and populations bit for bit
(bit-packed, packed bytes, plain bytes, Potts)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402


def result(cfg):
    r = eng.PARun(cfg)
    r.run()
    out = (r.rows(), r.population(), r.launch_shape())
    r.close()
    return out


CASES = [
    # config, other explicit shapes (group_threads, block_warps)
    (dict(L=16, R=1000, theta=5, beta_f=0.3, dbeta=0.05, seed=31, spin_format=eng.SPIN_BITS32),
     [(4, 8), (32, 2), (8, 4)]),
    (dict(L=32, R=700, theta=3, beta_f=0.2, dbeta=0.05, seed=32, spin_format=eng.SPIN_INT8),
     [(16, 8), (32, 4), (2, 2)]),
    (dict(L=6, R=500, theta=3, beta_f=0.3, dbeta=0.1, seed=33, spin_format=eng.SPIN_INT8),
     [(1, 8), (4, 2)]),
    (dict(L=16, R=400, theta=3, beta_f=0.6, dbeta=0.2, seed=34, spin_format=eng.SPIN_INT8, potts_q=3),
     [(2, 8), (32, 4)]),
]


@pytest.mark.parametrize("kw,others", CASES, ids=["bits", "packed-bytes", "bytes", "potts"])
def test_tuned_shape_used_and_results_unchanged(kw, others, tmp_path):
    path = str(tmp_path / "tune.txt")
    cfg = eng.PAConfig(**kw)
    ch = eng.autotune(cfg, cache_path=path)
    assert ch["candidates"] > 0 and ch["attempts_per_ns"] > 0
    key = eng.tune_key(cfg)
    assert eng.tune_cache_lookup(path, key)["group_threads"] == ch["group_threads"]
    again = eng.autotune(cfg, cache_path=path)  # remembered: no probes
    assert again["candidates"] == 0 and again["group_threads"] == ch["group_threads"]
    rows, pop, shape = result(cfg)  # shape left open: the tuned one
    assert shape["group_threads"] == ch["group_threads"]
    if ch["group_threads"] <= 32 and ch["block_warps"]:
        assert shape["block_threads"] <= 32 * ch["block_warps"]
    for g, bw in others:
        rows2, pop2, shape2 = result(eng.PAConfig(**kw, group_threads=g, block_warps=bw))
        assert shape2["group_threads"] == g
        np.testing.assert_array_equal(rows2, rows, err_msg=f"shape {g},{bw}")
        np.testing.assert_array_equal(pop2, pop, err_msg=f"shape {g},{bw}")


def test_cache_file_read_by_a_fresh_key(tmp_path):
    # a choice written for this device's key is found without probing
    path = str(tmp_path / "tune.txt")
    cfg = eng.PAConfig(L=8, R=3000, theta=2, beta_f=0.1, dbeta=0.05, seed=5, spin_format=eng.SPIN_BITS32)
    eng.tune_cache_store(path, eng.tune_key(cfg), {"group_threads": 4, "block_warps": 2, "attempts_per_ns": 1.0})
    ch = eng.autotune(cfg, cache_path=path)
    assert ch == {"group_threads": 4, "block_warps": 2, "attempts_per_ns": 1.0, "candidates": 0}
    rows, pop, shape = result(cfg)
    assert shape["group_threads"] == 4 and shape["block_threads"] == 64
    rows2, pop2, _ = result(eng.PAConfig(**{**cfg.__dict__, "group_threads": 1}))
    np.testing.assert_array_equal(rows2, rows)
    np.testing.assert_array_equal(pop2, pop)
