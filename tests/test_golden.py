"""Stored values under tests/golden/: the numbers the paper prints (cited in
paper_values.txt) are the ones the oracle and the bench use, and the
oracle-derived fixtures (written by tests/golden/make_golden.py, which
calls only oracle/) are reproduced exactly by the current oracle."""
import math
import random

import numpy as np
import pytest

from oracle import core
from oracle.exact_ising import BETA_C, BruteForce, potts_transfer_dos, transfer_matrix_dos
from oracle.pa_oracle import PopulationAnnealing, philox4x32_10
from tests.golden.make_golden import RUNS, ROW_FIELDS, fnv1a64, read_dos, read_paper_values, read_rows

PAPER = read_paper_values()


def test_beta_c_is_the_printed_formula():
    assert PAPER["beta_c_expr"] == "0.5*log(1+sqrt(2))"
    assert BETA_C == 0.5 * math.log(1.0 + math.sqrt(2.0))


def test_oracle_msc_words_follow_the_printed_lcg():
    """Sec. 4: each Philox word seeds r_{n+1} = A r_n + C mod 2^32; replica
    bit j of a word uses r_{j+1}. Checked against the oracle's MSC words
    with A and C as printed."""
    A, C, m = int(PAPER["lcg_A"]), int(PAPER["lcg_C"]), 1 << int(PAPER["lcg_modulus_log2"])
    rng = random.Random(5)
    for _ in range(200):
        seed = rng.getrandbits(64)
        u, c, b, k = rng.getrandbits(20), rng.getrandbits(1), rng.getrandbits(16), rng.getrandbits(20)
        r = philox4x32_10((2 * u + c, b >> 2, 5, k >> 5), (seed & 0xFFFFFFFF, seed >> 32))[b & 3]
        for _ in range((k & 31) + 1):
            r = (A * r + C) % m
        assert core().oracle_msc_word(seed, u, c, b, k) == r


def test_bench_default_workload_is_the_papers_default_run():
    import bench
    wl = bench.DEFAULT_WL
    assert wl["L"] == int(PAPER["default_L"]) and wl["theta"] == int(PAPER["default_theta"])
    assert wl["R"] == int(PAPER["default_R"]) and wl["beta_f"] == float(PAPER["default_beta_f"])
    assert wl["dbeta"] == float(PAPER["default_dbeta"]) and float(PAPER["default_beta0"]) == 0.0
    n_steps = round(wl["beta_f"] / wl["dbeta"])
    attempts = wl["L"] ** 2 * wl["theta"] * n_steps * wl["R"]
    assert bench.PAPER_K80_MSC_FLIPS_PER_NS == pytest.approx(attempts / float(PAPER["k80_seconds_msc"]) / 1e9,
                                                             rel=1e-15)


def test_exact_dos_fixture_reproduced():
    dos = read_dos()
    assert dos["square L=4 (enumeration)"] == BruteForce(4).energy_dos()
    assert dos["square L=6 (transfer matrix)"] == transfer_matrix_dos(6)
    assert dos["cubic L=2 (enumeration)"] == BruteForce(2, dim=3).energy_dos()
    assert dos["potts q=3 L=4 (transfer matrix)"] == potts_transfer_dos(4, 3)
    assert sum(dos["square L=6 (transfer matrix)"].values()) == 2 ** 36


@pytest.mark.parametrize("name", sorted(RUNS))
def test_oracle_rows_fixture_reproduced(name):
    params, h, rows = read_rows(name)
    p = RUNS[name]
    assert {k: params[k] for k in p} == p
    pa = PopulationAnnealing(p["L"], p["R"], p["theta"], beta_f=p["beta_f"], dbeta=p["dbeta"], seed=p["seed"],
                             dim=p["dim"], potts_q=p.get("potts_q", 0))
    pa.run()
    assert len(pa.rows) == len(rows)
    for got, ref in zip(pa.rows, rows):
        for k in ROW_FIELDS:
            assert getattr(got, k) == ref[k], (name, k)
    assert fnv1a64(pa.pop) == h
    assert np.all(np.array([r["R"] for r in rows]) > 0)
