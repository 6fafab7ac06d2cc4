"""Pins for the oracle's q-state Potts model (a further model the paper's
conclusion names; H = -sum over bonds of delta(s_i, s_j), Metropolis with a
uniform proposal of another state, dE = n(s) - n(s') for n(t) neighbours in
state t).

Independent facts: for q = 2 the model is the Ising model with
E_Potts = E_Ising/2 - N, so its counts are the Ising ones and Z_Potts(b) =
e^{bN} Z_Ising(b/2) (Kaufman); the transfer-matrix density of states equals
enumeration and has the hand-counted low levels (q ground states, none with
1..3 broken bonds, q(q-1)N with 4); a zero-temperature q = 2 sweep is the
Ising one; an always-accept sweep moves every site; zero-temperature sweeps
never raise the energy; PA rows against enumeration (q = 2 and 3) and the
exact q = 3 density of states; reweighting sums to q^N.
"""
import math

import numpy as np
import pytest

from oracle.exact_ising import (BruteForce, kaufman_lnZ, kaufman_observables, potts_averages, potts_enumerate,
                                potts_transfer_dos)
from oracle.pa_oracle import (PopulationAnnealing, init_spins, measure, measure_potts, sweep, sweep_potts)


def test_q2_counts_are_the_ising_counts():
    joint = potts_enumerate(4, 2)
    g = {}
    for (e, _), c in joint.items():
        g[e] = g.get(e, 0) + c
    assert g == {ei // 2 - 16: c for ei, c in BruteForce(4).energy_dos().items()}
    assert potts_transfer_dos(4, 2) == g


@pytest.mark.parametrize("q", [3, 4])
def test_transfer_dos_low_levels(q):
    g = potts_transfer_dos(4, q)
    N = 16
    assert sum(g.values()) == q ** N
    assert g[-2 * N] == q
    assert all(-2 * N + d not in g for d in (1, 2, 3))  # a domain costs at least 4 bonds
    assert g[-2 * N + 4] == q * (q - 1) * N            # one site in another state


def test_q2_lnZ_is_kaufman_at_half_beta():
    g = potts_transfer_dos(4, 2)
    E = np.array(list(g), dtype=np.float64)
    lg = np.log(np.array(list(g.values()), dtype=np.float64))
    for b in (0.3, 0.8, 1.5):
        lw = lg - b * E
        m = lw.max()
        assert m + math.log(float(np.exp(lw - m).sum())) == pytest.approx(16 * b + kaufman_lnZ(4, b / 2), rel=1e-12)


def test_zero_temperature_q2_sweep_is_the_ising_one():
    slots = np.arange(6, dtype=np.int64)
    sp = init_spins(8, slots, seed=9, potts_q=2)
    si = (1 - 2 * sp.astype(np.int16)).astype(np.int8)  # state 0 <-> +1, 1 <-> -1
    sweep_potts(sp, slots, 9, 0, 2, 2, (0, 0, 0, 0))
    sweep(si, slots, 9, 0, 2, 0, 0)
    np.testing.assert_array_equal(1 - 2 * sp.astype(np.int16), si)


def test_zero_temperature_never_raises_the_energy():
    slots = np.arange(8, dtype=np.int64)
    s = init_spins(8, slots, seed=11, potts_q=5)
    E0, _ = measure_potts(s, 5)
    for u in range(4):
        sweep_potts(s, slots, 11, u, 1, 5, (0, 0, 0, 0))
        E1, _ = measure_potts(s, 5)
        assert np.all(E1 <= E0)
        E0 = E1
    assert np.all((s >= 0) & (s < 5))


def test_always_accept_moves_every_site():
    slots = np.arange(4, dtype=np.int64)
    s = init_spins(6, slots, seed=13, potts_q=3)
    before = s.copy()
    sweep_potts(s, slots, 13, 0, 1, 3, (2 ** 32,) * 4)
    assert np.all(s != before) and np.all((s >= 0) & (s < 3))


def test_initial_states_are_uniform():
    s = init_spins(16, np.arange(200, dtype=np.int64), seed=17, potts_q=3)
    counts = np.bincount(s.ravel(), minlength=3)
    n = s.size
    chi2 = float(((counts - n / 3) ** 2 / (n / 3)).sum())
    assert chi2 < 20  # 2 degrees of freedom


COLS = ("e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N")


@pytest.mark.parametrize("L,q", [(4, 2), (2, 3)])
def test_rows_against_enumeration(L, q):
    exact = potts_enumerate(L, q)
    res = []
    for seed in range(400, 406):
        pa = PopulationAnnealing(L, 3000, 10, beta_f=2.0, dbeta=0.1, seed=seed, potts_q=q)
        pa.run()
        res.append([[getattr(r, c) for c in ("beta",) + COLS] for r in pa.rows])
    res = np.array(res)
    worst = 0.0
    for i in range(1, res.shape[1]):
        ex = potts_averages(exact, res[0, i, 0], L * L)
        for j, name in enumerate(COLS, start=1):
            mean = res[:, i, j].mean()
            se = res[:, i, j].std(ddof=1) / math.sqrt(res.shape[0])
            z = abs(mean - ex[name]) / (se + 2e-4)
            worst = max(worst, z)
            assert z < 8, (L, q, res[0, i, 0], name, mean, ex[name], se)
    assert worst > 0.1


def test_q2_L8_against_kaufman():
    """e_Potts(b) = e_Ising(b/2)/2 - 1, C_Potts(b) = C_Ising(b/2),
    beta F/N = -b + beta F_Ising(b/2)/N."""
    pa = PopulationAnnealing(8, 3000, 10, beta_f=1.6, dbeta=0.1, seed=19, potts_q=2)
    pa.run()
    for r in pa.rows[2::3]:
        ex = kaufman_observables(8, r.beta / 2)
        assert r.e == pytest.approx(ex["e"] / 2 - 1, abs=0.01), r.beta
        assert r.betaF_per_N == pytest.approx(-r.beta + ex["betaF_per_N"], abs=2e-3), r.beta


def test_q3_L4_energy_free_energy_and_dos():
    g = potts_transfer_dos(4, 3)
    E = np.array(list(g), dtype=np.float64)
    lg = np.log(np.array(list(g.values()), dtype=np.float64))
    pa = PopulationAnnealing(4, 4000, 10, beta_f=1.5, dbeta=0.1, seed=21, potts_q=3)
    pa.run()
    for r in pa.rows[1:]:
        lw = lg - r.beta * E
        m = lw.max()
        w = np.exp(lw - m)
        assert r.e == pytest.approx(float((w * E).sum() / w.sum()) / 16, abs=0.02), r.beta
        assert r.betaF_per_N == pytest.approx(-(m + math.log(float(w.sum()))) / 16, abs=3e-3), r.beta
    Ek, lno = pa.ln_dos()
    ok = np.isfinite(lno)
    mm = lno[ok].max()
    assert mm + math.log(float(np.exp(lno[ok] - mm).sum())) == pytest.approx(16 * math.log(3.0), abs=0.05)
    for k in np.nonzero(pa.Hsum >= 2000)[0]:
        assert lno[k] == pytest.approx(math.log(g[int(Ek[k])]), abs=0.1), int(Ek[k])
