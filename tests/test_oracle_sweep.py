"""Pins for the oracle's lattice, energy and Metropolis sweep (Sec. 2.1 step
3, Sec. 3 "Spin updates", Eq. hamiltonian).

Independent statements used here: the energy and the neighbour sums written
with ``np.roll`` on the 2D lattice, a zero-temperature greedy dynamics and an
always-accept dynamics that need no random numbers, and the exact Boltzmann
energy distribution of the 4 x 4 torus by enumeration.
"""
import math

import numpy as np
import pytest

from oracle.exact_ising import BruteForce
from oracle.pa_oracle import init_spins, measure, metropolis_threshold, sweep


def roll_energy(s):
    s = s.astype(np.int64)
    return (-(s * np.roll(s, -1, axis=-1)).sum(axis=(-1, -2))
            - (s * np.roll(s, -1, axis=-2)).sum(axis=(-1, -2)))


def aligned_count(s):
    s = s.astype(np.int64)
    nb = (np.roll(s, 1, -1) + np.roll(s, -1, -1) + np.roll(s, 1, -2) + np.roll(s, -1, -2))
    return (s * nb + 4) // 2  # s*nb = 2n - 4


def colour_mask(L):
    y, x = np.indices((L, L))
    return (x + y) & 1


@pytest.mark.parametrize("L", [4, 6, 8, 16])
def test_measure_matches_roll(L):
    s = init_spins(L, np.arange(50), 3)
    E, M = measure(s)
    np.testing.assert_array_equal(E, roll_energy(s))
    np.testing.assert_array_equal(M, s.astype(np.int64).sum(axis=(1, 2)))
    N = L * L
    assert np.all((E + 2 * N) % 4 == 0) and np.all((M + N) % 2 == 0)


def test_init_is_fair_and_slot_keyed():
    s = init_spins(16, np.arange(400), 11)
    frac = float((s > 0).mean())
    assert abs(frac - 0.5) < 5 * 0.5 / math.sqrt(s.size)
    # a replica's spins depend on its slot only, not on its position in the batch
    t = init_spins(16, np.array([399, 7]), 11)
    np.testing.assert_array_equal(t[0], s[399])
    np.testing.assert_array_equal(t[1], s[7])


@pytest.mark.parametrize("L", [4, 6, 8, 12, 16])
def test_zero_temperature_greedy(L):
    """Thresholds 0: only flips with dE <= 0 happen, deterministically.
    Reference: colour 0 then colour 1, each by a vectorised 2D rule."""
    s = init_spins(L, np.arange(20), 5)
    ref = s.astype(np.int64).copy()
    col = colour_mask(L)
    for _ in range(3):
        for c in (0, 1):
            n = aligned_count(ref)
            flip = (col == c) & (n <= 2)
            ref = np.where(flip, -ref, ref)
    got = s.copy()
    sweep(got, np.arange(20), 9, 0, 3, 0, 0)
    np.testing.assert_array_equal(got, ref.astype(np.int8))


@pytest.mark.parametrize("L", [4, 8, 16])
def test_always_accept_negates(L):
    """Thresholds 2^32: every site flips, so one sweep maps s -> -s."""
    s = init_spins(L, np.arange(10), 6)
    got = s.copy()
    sweep(got, np.arange(10), 9, 0, 1, 2 ** 32, 2 ** 32)
    np.testing.assert_array_equal(got, -s)
    sweep(got, np.arange(10), 9, 1, 1, 2 ** 32, 2 ** 32)
    np.testing.assert_array_equal(got, s)


def test_thresholds():
    assert metropolis_threshold(0.0, 4) == 2 ** 32
    b = 0.3
    t4 = metropolis_threshold(b, 4)
    assert (t4 - 1) / 2 ** 32 < math.exp(-4 * b) <= t4 / 2 ** 32
    assert metropolis_threshold(b, 8) < t4


@pytest.mark.parametrize("beta", [0.25, 0.44, 0.7])
def test_metropolis_samples_boltzmann_4x4(beta):
    """Independent chains from random starts, 60 sweeps each at fixed beta:
    the final energies follow the exact P(E) of the 4 x 4 torus (chi^2)."""
    L, n = 4, 6000
    s = init_spins(L, np.arange(n), 21)
    T4 = metropolis_threshold(beta, 4)
    T8 = metropolis_threshold(beta, 8)
    sweep(s, np.arange(n), 77, 0, 60, T4, T8)
    E, _ = measure(s)
    pmf = BruteForce(L).boltzmann_energy_pmf(beta)
    levels = sorted(pmf)
    obs = np.array([(E == e).sum() for e in levels], dtype=float)
    exp = np.array([pmf[e] * n for e in levels])
    keep = exp >= 5
    rest_o, rest_e = obs[~keep].sum(), exp[~keep].sum()
    o = np.append(obs[keep], rest_o)
    e = np.append(exp[keep], rest_e)
    if e[-1] < 5:
        o, e = o[:-1], e[:-1]
    chi2 = float(((o - e) ** 2 / e).sum())
    dof = len(o) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)
    assert obs.sum() == n


def test_swapped_thresholds_are_detected():
    """A planted mistake (T4 and T8 exchanged) must fail the Boltzmann check."""
    beta, L, n = 0.44, 4, 6000
    s = init_spins(L, np.arange(n), 21)
    sweep(s, np.arange(n), 77, 0, 60, metropolis_threshold(beta, 8), metropolis_threshold(beta, 4))
    E, _ = measure(s)
    pmf = BruteForce(L).boltzmann_energy_pmf(beta)
    mean_exact = sum(e * p for e, p in pmf.items())
    assert abs(E.mean() - mean_exact) > 10 * E.std() / math.sqrt(n)
