"""Pins for the oracle's population-annealing step (Sec. 2.1, Eq. Q,
Eq. resampling-factors, Eq. observables, Eq. free-energy, Eq. entropy).

What fixes the values independently of the oracle: the exact beta = 0 row
(Z_beta0 = 2^N), exact canonical averages of the 4 x 4 torus by
enumeration, Kaufman's ln Z for larger tori, the algebraic identities
sum_j tau_hat_j = R and R_i = sum_j r_j, Q written directly from Eq. Q, and
the binomial law of the nearest-integer copy numbers.
"""
import math

import numpy as np
import pytest

from oracle.exact_ising import BruteForce, kaufman_lnZ, kaufman_observables
from oracle.pa_oracle import (OracleError, PopulationAnnealing, copy_tables, level_weights,
                              normaliser_S, pairwise_sum, resample_words)


def test_row0_exact():
    pa = PopulationAnnealing(8, 500, 5, beta_f=0.1, dbeta=0.05, seed=4)
    r0 = pa.rows[0]
    assert r0.beta == 0.0 and r0.lnQ == 0.0 and r0.R == 500 and r0.families == 500
    assert r0.betaF_per_N == -math.log(2.0)
    assert r0.S_per_N == math.log(2.0) + 0.0 * r0.e  # beta * e = 0 at beta = 0


def test_pairwise_sum_is_a_sum():
    rng = np.random.default_rng(0)
    a = rng.random(1024)
    assert pairwise_sum(a) == pytest.approx(math.fsum(a), rel=1e-14)
    b = np.zeros(16)
    b[3] = 2.5
    assert pairwise_sum(b) == 2.5


def test_copy_tables_sum_to_R():
    rng = np.random.default_rng(1)
    N = 256
    H = np.zeros(N + 1, dtype=np.int64)
    H[40:90] = rng.integers(0, 50, 50)
    kmin, kmax = 40, 89
    for delta in [0.0, 0.01, 0.1, 0.7]:
        t = level_weights(delta, kmax - kmin + 1)
        S = normaliser_S(H, kmin, kmax, t, N)
        tau, F, U = copy_tables(1000, t, S)
        total = float((H[kmin:kmax + 1] * tau).sum())
        assert total == pytest.approx(1000.0, rel=1e-12)
        assert np.all(F >= 0) and np.all(U >= 0) and np.all(U <= 2 ** 32)


def test_identity_resampling_at_zero_step():
    # delta = 0 and R_{i-1} = R: tau_hat = 1, so every replica gets one copy
    N = 64
    H = np.zeros(N + 1, dtype=np.int64)
    H[10], H[20] = 300, 700
    t = level_weights(0.0, 11)
    S = normaliser_S(H, 10, 20, t, N)
    _, F, U = copy_tables(1000, t, S)
    assert S == 1000.0 and np.all(F == 1) and np.all(U == 0)


def test_single_replica_population_is_kept():
    """R = 1: one occupied level, S = t[0] = 1 and tau_hat = R t / S = 1
    exactly, so every step copies the one replica once (Eq. tau with
    R_{i-1} = R = 1); the population never grows, dies or splits."""
    pa = PopulationAnnealing(16, 1, 3, beta_f=0.5, dbeta=0.1, seed=21)
    pa.run()
    assert [r.R for r in pa.rows] == [1] * 6
    assert all(r.families == 1 for r in pa.rows)
    # Eq. Q with one replica: Q_i = exp(-dbeta E_{i-1}) exactly
    for prev, r in zip(pa.rows[:-1], pa.rows[1:]):
        assert r.lnQ == pytest.approx(-0.1 * prev.e * 256, rel=1e-12, abs=1e-12)


def test_copy_number_law():
    """r_j in {floor, floor+1} with Pr[floor+1] = frac(tau_hat): check the
    empirical frequency over many independent resampling streams."""
    frac_target = 0.3
    tau = 2.0 + frac_target
    U = math.ceil((tau - math.floor(tau)) * 2 ** 32)
    hits = 0
    n = 0
    for step in range(1, 41):
        x = resample_words(99, step, 1000).astype(np.int64)
        hits += int((x < U).sum())
        n += x.size
    p = hits / n
    assert abs(p - frac_target) < 5 * math.sqrt(frac_target * (1 - frac_target) / n)


def test_lnQ_matches_direct_definition():
    pa = PopulationAnnealing(8, 300, 3, beta_f=1.0, dbeta=0.1, seed=8)
    for _ in range(4):
        E_prev = pa.E.copy()
        rec = pa.step()
        q = math.fsum(math.exp(-rec.delta * float(e)) for e in E_prev) / E_prev.size
        assert rec.lnQ == pytest.approx(math.log(q), rel=1e-12, abs=1e-13)


def test_invariants_along_a_run():
    pa = PopulationAnnealing(8, 700, 4, beta_f=1.0, dbeta=0.05, seed=12)
    pa.run()
    N = pa.N
    fam_prev = None
    for i, rec in enumerate(pa.records):
        assert rec.H_E.sum() == rec.R and rec.H_M.sum() == rec.R
        if i > 0:
            assert rec.counts.sum() == rec.R
            assert rec.counts.size == pa.records[i - 1].R
            assert np.all(np.diff(rec.parent) >= 0)  # copies follow old-slot order
            assert rec.families <= fam_prev
        fam_prev = rec.families
    assert np.all((pa.E + 2 * N) % 4 == 0)
    assert pa.rows[-1].beta == pytest.approx(1.0, abs=1e-15)
    assert len(pa.rows) == 21


def test_deterministic():
    a = PopulationAnnealing(8, 200, 3, beta_f=0.3, dbeta=0.1, seed=5)
    b = PopulationAnnealing(8, 200, 3, beta_f=0.3, dbeta=0.1, seed=5)
    a.run()
    b.run()
    np.testing.assert_array_equal(a.pop, b.pop)
    assert [r.as_tuple() for r in a.rows] == [r.as_tuple() for r in b.rows]


def test_capacity_error():
    pa = PopulationAnnealing(8, 500, 1, beta_f=1.0, dbeta=0.2, seed=3, capacity=500)
    with pytest.raises(OracleError) as ei:
        pa.run()
    assert ei.value.kind == "capacity"


def test_extinction_only_when_every_copy_weight_is_below_one():
    """Sec. 2.1, Eq. resampling-factors: replica j expects
    tau_j = R exp(-dbeta E_j) / sum_l exp(-dbeta E_l) copies, at least one of
    which is at least 1 when R_{i-1} <= R; so a population can die out only
    after it has grown past R and every tau_j is below 1. With L = 8, R = 2,
    theta = 1, dbeta = 0.05 and seed 113 it dies out at step 3; the expected
    copy numbers of the population it resampled are written out here from the
    equation (numpy exp and sum, not the oracle's tables)."""
    pa = PopulationAnnealing(8, 2, 1, beta_f=1.0, dbeta=0.05, seed=113)
    with pytest.raises(OracleError) as ei:
        pa.run()
    assert ei.value.kind == "extinct"
    assert len(pa.records) == 3 and len(pa.rows) == 3  # steps 0, 1, 2 completed
    E = pa.E.astype(np.float64)  # energies of population 2, the one step 3 resampled
    assert E.size > 2 and E.size == pa.records[-1].R
    w = np.exp(-0.05 * (E - E.min()))
    tau = 2.0 * w / w.sum()
    assert tau.max() < 1.0
    # the same run with more replicas does not die out
    big = PopulationAnnealing(8, 8, 1, beta_f=1.0, dbeta=0.05, seed=113)
    big.run()
    assert big.done


def _runs(L, R, theta, dbeta, seeds):
    out = []
    for s in seeds:
        pa = PopulationAnnealing(L, R, theta, beta_f=1.0, dbeta=dbeta, seed=s)
        pa.run()
        out.append(np.array([r.as_tuple() for r in pa.rows]))
    return np.array(out)


COLS = {"e": 1, "C": 2, "abs_m": 3, "m2": 4, "m4": 5, "betaF_per_N": 6, "S_per_N": 7}


def test_4x4_against_enumeration():
    """Six independent runs; each observable at each beta within 8 standard
    errors (plus a small allowance for the O(1/R) bias of PA)."""
    res = _runs(4, 4000, 10, 0.05, range(100, 106))
    bf = BruteForce(4)
    worst = 0.0
    for i in range(1, res.shape[1]):
        beta = res[0, i, 0]
        ex = bf.averages(beta)
        for name, c in COLS.items():
            mean = res[:, i, c].mean()
            se = res[:, i, c].std(ddof=1) / math.sqrt(res.shape[0])
            z = abs(mean - ex[name]) / (se + 2e-4)
            worst = max(worst, z)
            assert z < 8, (beta, name, mean, ex[name], se)
    assert worst > 0.1  # the comparison is not vacuous


def test_8x8_against_kaufman():
    res = _runs(8, 3000, 10, 0.05, range(200, 204))
    for i in [2, 6, 9, 12, 16, 20]:
        beta = res[0, i, 0]
        ex = kaufman_observables(8, beta)
        for name in ("e", "C", "betaF_per_N", "S_per_N"):
            c = COLS[name]
            mean = res[:, i, c].mean()
            se = res[:, i, c].std(ddof=1) / math.sqrt(res.shape[0])
            assert abs(mean - ex[name]) < 8 * (se + 2e-4), (beta, name, mean, ex[name], se)


def test_free_energy_sign_and_scale():
    # a planted sign error in ln Q would move beta F/N by ~2 sum ln Q / N;
    # at beta = 1 on 8 x 8 the exact value is fixed by Kaufman to 1e-3
    pa = PopulationAnnealing(8, 2000, 10, beta_f=1.0, dbeta=0.05, seed=31)
    pa.run()
    ex = -kaufman_lnZ(8, 1.0) / 64
    assert pa.rows[-1].betaF_per_N == pytest.approx(ex, abs=3e-3)
