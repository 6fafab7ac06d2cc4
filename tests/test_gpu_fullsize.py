"""Full-size checks on the configurations of the paper's workloads, in the
launch configuration bench.py times.

Step-by-step parity at full population: the oracle's block-parallel form
(bit-identical to its serial form) runs the first steps of config 2 (L=64,
R=20000, theta=100, dbeta=0.005, seed 2) and config 3 (L=128, R=50000,
theta=50, adaptive overlap 0.85, seed 3) beside the engine; after every step
the whole population, every energy, magnetisation and family, both
histograms, R_i, S, the step size, the thresholds and the row must agree.

Sampled parity: the oracle computes step 1 from scratch (all initial spins
and energies, every copy number, the parents) and sweeps only sampled new
slots; the GPU's spins, energies and families of those slots must match
bit for bit, and R_1, S and the step-0 histogram exactly.

Properties of whole runs (no oracle run needed): histogram sums, energies
recomputed from the final spins, the exact beta = 0 row, and agreement with
Kaufman's exact finite-lattice results within statistical error.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from oracle.exact_ising import kaufman_lnZ, kaufman_observables  # noqa: E402
from oracle.pa_oracle import PopulationAnnealing  # noqa: E402

B32 = eng.SPIN_BITS32


def roll_energy(s):
    s = s.astype(np.int64)
    return -(s * np.roll(s, -1, -1)).sum(axis=(-1, -2)) - (s * np.roll(s, -1, -2)).sum(axis=(-1, -2))


def sampled_step1(L, R, theta, dbeta, seed, nsample=24):
    pa = PopulationAnnealing(L, R, theta, beta_f=1.0, dbeta=dbeta, seed=seed, record_hist=True)
    run = eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, beta_f=1.0, dbeta=dbeta, seed=seed, spin_format=B32,
                                 record_histograms=True))
    np.testing.assert_array_equal(run.histogram(0, 0), pa.records[0].H_E)
    assert run.step()
    info = run.step_info(1)
    rng = np.random.default_rng(seed)
    chosen = {}

    def pick(R1):  # R_1 is known only after the oracle's resampling
        chosen["s"] = np.unique(np.concatenate([[0, 1, R1 - 1], rng.integers(0, R1, nsample)]))
        return chosen["s"]

    rec2 = pa.step(sample=pick)
    sample = chosen["s"]
    assert info["R"] == rec2.R and info["S"] == rec2.S and info["delta"] == rec2.delta
    pa2 = pa
    pop = run.population()
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(pop[sample], rec2.sample_pop)
    np.testing.assert_array_equal(E[sample], rec2.sample_E)
    np.testing.assert_array_equal(M[sample], rec2.sample_M)
    np.testing.assert_array_equal(fam[sample], rec2.sample_fam)
    # the whole family vector follows from the parents alone
    np.testing.assert_array_equal(fam, pa2.fam[rec2.parent])
    assert run.rows()[1]["families"] == np.unique(pa2.fam[rec2.parent]).size
    run.close()


def test_config2_step1_sampled_parity():
    """L=64, R=20000, theta=100, dbeta=0.005, seed 2 (the bench workload)."""
    sampled_step1(64, 20000, 100, 0.005, 2)


def test_config3_step1_sampled_parity():
    """L=128, R=50000, theta=50, adaptive overlap 0.85, seed 3."""
    sampled_step1(128, 50000, 50, 0.0, 3, nsample=12)


def stepwise_fullsize(L, R, theta, dbeta, seed, n_steps):
    from tests._parity import assert_row_close, compare_step
    pa = PopulationAnnealing(L, R, theta, beta_f=1.0, dbeta=dbeta, seed=seed, overlap=0.85, record_hist=True,
                             workers=os.cpu_count() or 1)
    run = eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, beta_f=1.0, dbeta=dbeta, overlap=0.85, seed=seed,
                                 spin_format=B32, record_histograms=True))

    def check(i):
        compare_step(run, pa, i)
        assert_row_close(run.rows()[i], pa.rows[i], f"row {i}")
        E, M, fam = run.replicas()
        np.testing.assert_array_equal(E, pa.E, err_msg=f"E step {i}")
        np.testing.assert_array_equal(M, pa.M, err_msg=f"M step {i}")
        np.testing.assert_array_equal(fam, pa.fam, err_msg=f"families step {i}")
        np.testing.assert_array_equal(run.population(), pa.pop, err_msg=f"spins step {i}")

    check(0)
    for i in range(1, n_steps + 1):
        assert run.step()
        pa.step()
        check(i)
    run.close()


def test_config2_first_10_steps_bit_exact():
    stepwise_fullsize(64, 20000, 100, 0.005, 2, 10)


def test_config3_first_5_steps_bit_exact():
    stepwise_fullsize(128, 50000, 50, 0.0, 3, 5)


def check_run_properties(run, L, R):
    N = L * L
    rows = run.rows()
    assert rows[0]["betaF_per_N"] == -math.log(2.0) and rows[0]["S_per_N"] == math.log(2.0)
    for i in range(len(rows)):
        info = run.step_info(i)
        assert rows[i]["R"] == info["R"]
        assert abs(info["R"] - R) < 12 * math.sqrt(R)
    pop = run.population()
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(E, roll_energy(pop))
    np.testing.assert_array_equal(M, pop.astype(np.int64).sum(axis=(1, 2)))
    H = run.histogram(len(rows) - 1, 0)
    assert H.sum() == rows[-1]["R"]
    np.testing.assert_array_equal(H, np.bincount((E + 2 * N) // 4, minlength=N + 1))
    assert np.all(np.diff(fam) >= 0)
    return rows


def test_config2_full_run_properties():
    run = eng.PARun(eng.PAConfig(L=64, R=20000, theta=100, beta_f=1.0, dbeta=0.005, seed=2, spin_format=B32))
    run.run()
    rows = check_run_properties(run, 64, 20000)
    assert len(rows) == 201
    for i in (20, 60, 88, 100, 140, 200):
        b = rows[i]["beta"]
        ex = kaufman_observables(64, b)
        assert abs(rows[i]["e"] - ex["e"]) < 2e-3, (b, rows[i]["e"], ex["e"])
        assert abs(rows[i]["betaF_per_N"] - ex["betaF_per_N"]) < 1e-3, (b,)
        assert abs(rows[i]["C"] - ex["C"]) < 0.05 * max(ex["C"], 0.2), (b, rows[i]["C"], ex["C"])
    run.close()


def test_config3_full_run_mhr():
    """Adaptive PA at L=128, R=50000, theta=50, then multi-histogram
    reweighting: ln Z(beta) and e(beta) against Kaufman."""
    run = eng.PARun(eng.PAConfig(L=128, R=50000, theta=50, beta_f=1.0, dbeta=0.0, overlap=0.85, seed=3,
                                 spin_format=B32))
    run.run()
    rows = check_run_properties(run, 128, 50000)
    assert 300 < len(rows) < 600 and rows[-1]["beta"] == 1.0
    betas = np.array([r["beta"] for r in rows])
    assert np.all(np.diff(betas) > 0)
    for b in (0.2, 0.4, 0.44, 0.5, 0.8):
        m = run.mhr([b])[0]
        assert abs(m["betaF_per_N"] + kaufman_lnZ(128, b) / 128 ** 2) < 5e-4, b
        assert abs(m["e"] - kaufman_observables(128, b)["e"]) < 5e-3, b
    run.close()
