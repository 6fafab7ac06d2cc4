"""Pins for combining M independent runs (Sec. 2.2, Eq. weighted-average)
and for reusing the first run's adaptive schedule (Sec. 2.3)."""
import math

import numpy as np
import pytest

from oracle.exact_ising import BruteForce, kaufman_lnZ
from oracle.pa_oracle import PopulationAnnealing, Row, weighted_average


def row(beta, N, e, C, betaF, R=100):
    return Row(beta, e, C, 0.5, 0.3, 0.1, betaF, beta * e - betaF, 0.0, R, 10, N)


def test_identical_runs_average_to_themselves():
    r = [row(0.3, 16, -0.7, 0.4, -0.8)]
    out = weighted_average([r, r, r])[0]
    assert out["weights"] == pytest.approx([1 / 3] * 3)
    assert out["e"] == pytest.approx(-0.7) and out["C"] == pytest.approx(0.4)
    assert out["betaF_per_N"] == pytest.approx(-0.8)  # ln((1/M) M Z) = ln Z
    assert out["R"] == 300


def test_two_runs_closed_form():
    # Z_B = 3 Z_A  =>  weights 1/4, 3/4; combined ln Z = ln(2 Z_A)
    N, beta = 16, 0.5
    a = row(beta, N, -1.0, 0.2, -1.0)
    b = row(beta, N, -1.2, 0.3, -1.0 - math.log(3.0) / N)
    out = weighted_average([[a], [b]])[0]
    assert out["weights"] == pytest.approx([0.25, 0.75], rel=1e-12)
    assert out["e"] == pytest.approx(0.25 * -1.0 + 0.75 * -1.2, rel=1e-12)
    e2 = 0.25 * (0.2 / (beta * beta * N) + 1.0) + 0.75 * (0.3 / (beta * beta * N) + 1.44)
    assert out["C"] == pytest.approx(beta * beta * N * (e2 - out["e"] ** 2), rel=1e-12)
    assert out["betaF_per_N"] == pytest.approx(-(N * 1.0 + math.log(2.0)) / N, rel=1e-12)


def test_mismatched_betas_rejected():
    with pytest.raises(ValueError):
        weighted_average([[row(0.3, 16, -1, 0, -1)], [row(0.31, 16, -1, 0, -1)]])


def test_weighted_runs_estimate_the_free_energy():
    """Eight small-population runs of the 4x4 torus: the combined free energy
    (the log of the mean partition-function estimate) sits within its
    statistical error of the exact value at every beta."""
    runs = []
    for s in range(8):
        pa = PopulationAnnealing(4, 200, 5, beta_f=1.0, dbeta=0.05, seed=500 + s)
        pa.run()
        runs.append(pa.rows)
    comb = weighted_average(runs)
    bf = BruteForce(4)
    for i in (4, 10, 20):
        b = comb[i]["beta"]
        ex = bf.averages(b)
        spread = np.std([rr[i].betaF_per_N for rr in runs], ddof=1)
        assert abs(comb[i]["betaF_per_N"] - ex["betaF_per_N"]) < 4 * spread / math.sqrt(8) + 1e-3
        assert abs(comb[i]["e"] - ex["e"]) < 0.05
        assert sum(comb[i]["weights"]) == pytest.approx(1.0)


def test_schedule_reuse():
    first = PopulationAnnealing(8, 800, 5, beta_f=0.6, dbeta=0.0, seed=41)
    first.run()
    sched = [r.beta for r in first.rows[1:]]
    second = PopulationAnnealing(8, 800, 5, beta_f=0.6, seed=42, schedule=sched)
    second.run()
    assert [r.beta for r in second.rows[1:]] == sched
    assert second.records[1].delta == sched[0]
    comb = weighted_average([first.rows, second.rows])
    ex = -kaufman_lnZ(8, 0.6) / 64
    assert abs(comb[-1]["betaF_per_N"] - ex) < 5e-3


def test_engine_weighted_average_matches_oracle():
    """pa_weighted_average is host code: it runs here, without a GPU, and
    must agree with the oracle's statement of Eq. weighted-average."""
    eng = pytest.importorskip("paper_1703_03676_gb300")
    runs = []
    for s in range(3):
        pa = PopulationAnnealing(4, 150, 3, beta_f=0.5, dbeta=0.1, seed=70 + s)
        pa.run()
        runs.append(pa.rows)
    ref = weighted_average(runs)
    dt = np.dtype([(f, np.float64) for f in ("beta", "e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N", "lnQ")]
                  + [("R", np.int64), ("families", np.int64)])
    arrs = []
    for rr in runs:
        a = np.zeros(len(rr), dtype=dt)
        for i, r in enumerate(rr):
            a[i] = r.as_tuple()
        arrs.append(a)
    got = eng.weighted_average(arrs, 16)
    for i, g in enumerate(ref):
        for f in ("beta", "e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N"):
            assert got[f][i] == pytest.approx(g[f], rel=1e-12, abs=1e-14), (i, f)
        assert got["R"][i] == g["R"] and got["families"][i] == g["families"]
