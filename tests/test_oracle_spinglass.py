"""Pins for the +-J (Edwards-Anderson) model: quenched couplings shared by
the population (the paper's method applies to disordered systems, Sec. 1).

Independent facts: enumeration with couplings; all couplings +1 reduce to
the ferromagnet; a gauge transformation (flip the spins of a set of sites
and the couplings around them) leaves energies invariant; the Metropolis
sweep samples the exact Boltzmann law of a 4 x 4 instance (chi^2); PA rows
and the ground state agree with enumeration."""
import math

import numpy as np
import pytest

from oracle.exact_ising import BruteForce, enumerate_states, enumerate_states_j
from oracle.pa_oracle import (PopulationAnnealing, init_spins, measure, metropolis_threshold, random_couplings,
                              sweep)


def test_all_plus_couplings_is_the_ferromagnet():
    ones = (np.ones((4, 4), np.int8), np.ones((4, 4), np.int8))
    E1, M1 = enumerate_states_j(4, *ones)
    E0, M0 = enumerate_states(4)
    np.testing.assert_array_equal(E1, E0)
    s = init_spins(8, np.arange(20), 3)
    np.testing.assert_array_equal(measure(s, (np.ones((8, 8), np.int8),) * 2)[0], measure(s)[0])


def test_gauge_invariance():
    L = 8
    Jr, Jd = random_couplings(L, 5)
    s = init_spins(L, np.arange(30), 9).astype(np.int64)
    g = np.where(np.random.default_rng(1).random((L, L)) < 0.5, -1, 1)
    Jr2 = (Jr * g * np.roll(g, -1, axis=1)).astype(np.int8)
    Jd2 = (Jd * g * np.roll(g, -1, axis=0)).astype(np.int8)
    E1, _ = measure(s.astype(np.int8), (Jr, Jd))
    E2, _ = measure((s * g).astype(np.int8), (Jr2, Jd2))
    np.testing.assert_array_equal(E1, E2)


def test_energy_levels_are_integral():
    Jr, Jd = random_couplings(6, 11)
    E, _ = measure(init_spins(6, np.arange(50), 1), (Jr, Jd))
    assert np.all((E + 72) % 4 == 0)


@pytest.mark.parametrize("beta", [0.3, 0.7, 1.2])
def test_sweep_samples_boltzmann_pm_j_4x4(beta):
    J = random_couplings(4, 21)
    n = 6000
    s = init_spins(4, np.arange(n), 23)
    sweep(s, np.arange(n), 91, 0, 80, metropolis_threshold(beta, 4), metropolis_threshold(beta, 8), couplings=J)
    E, _ = measure(s, J)
    pmf = BruteForce(4, J).boltzmann_energy_pmf(beta)
    levels = sorted(pmf)
    obs = np.array([(E == e).sum() for e in levels], dtype=float)
    exp = np.array([pmf[e] * n for e in levels])
    keep = exp >= 5
    o = np.append(obs[keep], obs[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] < 5:
        o, e = o[:-1], e[:-1]
    chi2 = float(((o - e) ** 2 / e).sum())
    dof = len(o) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)
    assert obs.sum() == n


def test_pa_spin_glass_against_enumeration():
    J = random_couplings(4, 33)
    bf = BruteForce(4, J)
    res = []
    for sd in range(6):
        pa = PopulationAnnealing(4, 3000, 10, beta_f=2.0, dbeta=0.1, seed=700 + sd, couplings=J)
        pa.run()
        res.append([r.as_tuple() for r in pa.rows])
    res = np.array(res)
    for i in (5, 10, 20):
        ex = bf.averages(res[0, i, 0])
        for name, c in (("e", 1), ("C", 2), ("betaF_per_N", 6)):
            mean = res[:, i, c].mean()
            se = res[:, i, c].std(ddof=1) / math.sqrt(6)
            assert abs(mean - ex[name]) < 8 * (se + 5e-4), (name, mean, ex[name])
    # at beta = 2 the population sits at the ground state of the instance
    e0 = min(bf.energy_dos()) / 16
    assert res[:, -1, 1].mean() == pytest.approx(e0, abs=0.02)
