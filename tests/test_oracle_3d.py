"""Pins for the oracle's simple cubic Ising model (the three-dimensional
model the paper's conclusion names as a further target of the method; the
update is the Metropolis rule of Sec. 3 with six neighbours, dE = 4n - 12).

Independent facts: the exact 2 x 2 x 2 density of states (enumeration) and
its hand counts; zero-temperature dynamics against an independent array
implementation; an always-accept sweep negates every spin; PA rows of the
2 x 2 x 2 torus against enumeration; the high-temperature expansion
ln Z / N = ln 2 + 3 ln cosh b + 3 t^4 + O(t^6) (t = tanh b; three plaquettes
per site) at L = 8; the low-temperature expansion e = -3 + 12 exp(-12 b)
+ ... at L = 4; the reweighted density of states summing to 2^N.
"""
import math

import numpy as np
import pytest

from oracle.exact_ising import BruteForce
from oracle.pa_oracle import PopulationAnnealing, init_spins, measure, sweep


def test_enumeration_2x2x2_counts():
    g = BruteForce(2, dim=3).energy_dos()
    N = 8
    assert sum(g.values()) == 2 ** N
    assert g[-3 * N] == 2                  # the two ground states
    assert -3 * N + 4 not in g and -3 * N + 8 not in g
    assert g[-3 * N + 12] == 2 * N         # one flipped spin breaks its 6 bonds
    assert all(g[e] == g[-e] for e in g)   # flipping one sublattice: E -> -E


def _greedy_reference(s):
    """One zero-temperature checkerboard sweep written with array shifts:
    colour 0 then colour 1, a site flips iff at most 3 of its 6 neighbours
    agree with it (dE <= 0)."""
    s = s.copy()
    L = s.shape[0]
    z, y, x = np.indices((L, L, L))
    colour = (x + y + z) & 1
    for c in (0, 1):
        nb = sum(np.roll(s, sh, axis=ax) for ax in (0, 1, 2) for sh in (1, -1))
        aligned = (6 + s * nb) // 2
        flip = (colour == c) & (aligned <= 3)
        s[flip] = -s[flip]
    return s


def test_zero_temperature_sweep_matches_array_rule():
    pop = init_spins(6, np.arange(5, dtype=np.int64), seed=3, dim=3)
    ref = np.array([_greedy_reference(p) for p in pop])
    sweep(pop, np.arange(5, dtype=np.int64), 3, 0, 1, 0, 0, T12=0)
    np.testing.assert_array_equal(pop, ref)


def test_always_accept_negates_every_spin():
    pop = init_spins(4, np.arange(3, dtype=np.int64), seed=5, dim=3)
    before = pop.copy()
    sweep(pop, np.arange(3, dtype=np.int64), 5, 0, 1, 2 ** 32, 2 ** 32, T12=2 ** 32)
    np.testing.assert_array_equal(pop, -before)


def test_measure_counts_three_bonds_per_site():
    up = np.ones((1, 4, 4, 4), dtype=np.int8)
    E, M = measure(up)
    assert E[0] == -3 * 64 and M[0] == 64
    stag = np.fromfunction(lambda z, y, x: 1 - 2 * ((x + y + z) % 2), (4, 4, 4), dtype=int).astype(np.int8)
    E, M = measure(stag[None])
    assert E[0] == 3 * 64 and M[0] == 0


COLS = ("e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N")


def test_rows_2x2x2_against_enumeration():
    bf = BruteForce(2, dim=3)
    res = []
    for seed in range(300, 306):
        pa = PopulationAnnealing(2, 4000, 10, beta_f=1.0, dbeta=0.05, seed=seed, dim=3)
        pa.run()
        res.append([[getattr(r, c) for c in ("beta",) + COLS] for r in pa.rows])
    res = np.array(res)
    worst = 0.0
    for i in range(1, res.shape[1]):
        ex = bf.averages(res[0, i, 0])
        for j, name in enumerate(COLS, start=1):
            mean = res[:, i, j].mean()
            se = res[:, i, j].std(ddof=1) / math.sqrt(res.shape[0])
            z = abs(mean - ex[name]) / (se + 2e-4)
            worst = max(worst, z)
            assert z < 8, (res[0, i, 0], name, mean, ex[name], se)
    assert worst > 0.1


def _high_t_lnZ_per_site(b):
    t = math.tanh(b)
    return math.log(2.0) + 3.0 * math.log(math.cosh(b)) + 3.0 * t ** 4


def test_high_temperature_expansion_L8():
    """At beta = 0.1 the next term (22 t^6 in ln Z / N on the simple cubic
    lattice) moves e by about 1.3e-3 and beta F / N by 2e-5; the t^4 term
    moves e by 1.2e-2, the t^2 difference to the square lattice by 0.1.
    Loops around the L = 8 torus enter at t^8. dbeta = 0.01 keeps
    dbeta * sigma_E ~ 0.4 (sigma_E ~ sqrt(3N)), so ln Q is unbiased to
    ~1e-5 per step."""
    pa = PopulationAnnealing(8, 6000, 5, beta_f=0.1, dbeta=0.01, seed=41, dim=3)
    pa.run()
    row = pa.rows[-1]
    b, h = 0.1, 1e-5
    e_series = -(_high_t_lnZ_per_site(b + h) - _high_t_lnZ_per_site(b - h)) / (2 * h)
    assert row.beta == pytest.approx(0.1, abs=1e-15)
    assert row.e == pytest.approx(e_series, abs=3e-3)
    assert row.betaF_per_N == pytest.approx(-_high_t_lnZ_per_site(b), abs=2e-4)


def test_low_temperature_expansion_L4():
    """Lowest excitations of the ordered state: one flipped spin costs 12,
    so e = -3 + 12 exp(-12 beta) + O(exp(-20 beta)) per site."""
    pa = PopulationAnnealing(4, 2000, 10, beta_f=1.0, dbeta=0.05, seed=43, dim=3)
    pa.run()
    row = pa.rows[-1]
    assert row.e == pytest.approx(-3.0 + 12.0 * math.exp(-12.0), abs=1e-3)
    assert row.abs_m == pytest.approx(1.0, abs=1e-3)


def test_reweighted_dos_sums_to_2_pow_N_and_matches_2x2x2():
    pa = PopulationAnnealing(2, 4000, 10, beta_f=1.0, dbeta=0.0, seed=47, dim=3)
    pa.run()
    E, lno = pa.ln_dos()
    ok = np.isfinite(lno)
    m = lno[ok].max()
    assert m + math.log(float(np.exp(lno[ok] - m).sum())) == pytest.approx(8 * math.log(2.0), abs=0.05)
    g = BruteForce(2, dim=3).energy_dos()
    for k in np.nonzero(pa.Hsum >= 2000)[0]:
        assert lno[k] == pytest.approx(math.log(g[int(E[k])]), abs=0.1), int(E[k])
