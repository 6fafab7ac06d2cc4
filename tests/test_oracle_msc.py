"""Pins for the multi-spin-coded variant (Sec. 4): 32 replicas per word,
their random numbers drawn from a Philox-seeded linear congruential
generator (A = 1664525, C = 1013904223, the paper's choice).

The paper's evidence that this variant is unbiased (Fig. 2, Table 1) is
statistical; here: the Boltzmann law of the 4 x 4 torus (chi^2), exact
PA observables, the same variance of C as the single-spin contract, the
LCG's full period, and that the 32 replicas of a word get distinct
numbers."""
import math

import numpy as np
import pytest

from oracle.exact_ising import BruteForce
from oracle.pa_oracle import PopulationAnnealing, init_spins, measure, metropolis_threshold, sweep


def test_lcg_constants_give_full_period():
    # Hull-Dobell: C odd, A - 1 divisible by 4 (and by 2, the only prime
    # factor of 2^32) => the LCG has the full period 2^32
    A, C = 1664525, 1013904223
    assert C % 2 == 1 and (A - 1) % 4 == 0


@pytest.mark.parametrize("beta", [0.3, 0.44, 0.7])
def test_msc_samples_boltzmann_4x4(beta):
    L, n = 4, 6400  # 200 words of 32 replicas
    s = init_spins(L, np.arange(n), 23)
    sweep(s, np.arange(n), 91, 0, 60, metropolis_threshold(beta, 4), metropolis_threshold(beta, 8), msc=True)
    E, _ = measure(s)
    pmf = BruteForce(L).boltzmann_energy_pmf(beta)
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


def test_msc_replicas_of_a_word_differ():
    """Identical copies in one word must evolve differently (a shared random
    number would keep them identical, the correlation Fig. 2 shows)."""
    L = 8
    one = init_spins(L, np.array([0]), 5)
    s = np.repeat(one, 32, axis=0).copy()
    sweep(s, np.arange(32), 7, 0, 5, metropolis_threshold(0.3, 4), metropolis_threshold(0.3, 8), msc=True)
    distinct = {bytes(x.tobytes()) for x in s}
    assert len(distinct) > 28


def _C_spread(msc, seeds):
    vals = []
    for sd in seeds:
        pa = PopulationAnnealing(8, 640, 5, beta_f=0.45, dbeta=0.05, seed=sd, msc=msc)
        pa.run()
        vals.append(pa.rows[-1].C)
    return np.mean(vals), np.var(vals, ddof=1)


def test_msc_variance_of_C_matches_single_spin():
    """Fig. 2 (c) and Table 1 (LCG rows: sigma^2_MSC(C)/sigma^2_SSC(C) = 1,
    tests/golden/paper_values.txt): the LCG variant leaves sigma^2(C)
    unchanged; 16 runs each bound the ratio within a factor 3."""
    from tests.golden.make_golden import read_paper_values
    ratio = float(read_paper_values()["msc_lcg_var_ratio_C"])
    m1, v1 = _C_spread(False, range(300, 316))
    m2, v2 = _C_spread(True, range(300, 316))
    assert ratio / 3 < v2 / v1 < ratio * 3
    assert abs(m1 - m2) < 4 * math.sqrt(v1 / 16 + v2 / 16)


def test_msc_pa_against_enumeration():
    res = []
    for sd in range(6):
        pa = PopulationAnnealing(4, 3200, 10, beta_f=1.0, dbeta=0.05, seed=400 + sd, msc=True)
        pa.run()
        res.append([r.as_tuple() for r in pa.rows])
    res = np.array(res)
    bf = BruteForce(4)
    for i in (4, 9, 14, 20):
        ex = bf.averages(res[0, i, 0])
        for name, c in (("e", 1), ("abs_m", 3), ("betaF_per_N", 6)):
            mean = res[:, i, c].mean()
            se = res[:, i, c].std(ddof=1) / math.sqrt(6)
            assert abs(mean - ex[name]) < 8 * (se + 2e-4), (name, mean, ex[name])
