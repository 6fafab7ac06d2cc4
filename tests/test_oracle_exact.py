"""Pins for the exact Ising references used to pin the oracle.

Three independent routes to ln Z of the periodic L x L Ising model must agree:
full enumeration (L = 4), the row transfer matrix (L <= 8) and Kaufman's
closed form (Sec. 3 notes that exact results exist for this model).
"""
import math

import numpy as np
import pytest

from oracle.exact_ising import (BETA_C, BruteForce, kaufman_lnZ, kaufman_observables,
                                transfer_matrix_dos, transfer_matrix_lnZ)

BETAS = [0.0, 0.05, 0.2, 0.4, BETA_C, 0.5, 0.8, 1.0, 1.5]


def test_beta_c_closed_form():
    # beta_c = ln(1 + sqrt 2)/2 (Sec. 3); sinh(2 beta_c) = 1 is the self-dual point
    assert math.isclose(math.sinh(2 * BETA_C), 1.0, rel_tol=1e-15)


@pytest.mark.parametrize("beta", BETAS)
def test_bruteforce_vs_transfer_vs_kaufman_L4(beta):
    bf = BruteForce(4)
    a = bf.lnZ(beta)
    assert math.isclose(a, transfer_matrix_lnZ(4, beta), rel_tol=1e-13)
    assert math.isclose(a, kaufman_lnZ(4, beta), rel_tol=1e-13)


@pytest.mark.parametrize("L", [6, 8])
@pytest.mark.parametrize("beta", [0.05, 0.3, BETA_C, 0.7, 1.2])
def test_transfer_vs_kaufman(L, beta):
    assert math.isclose(transfer_matrix_lnZ(L, beta), kaufman_lnZ(L, beta), rel_tol=1e-12)


def test_bruteforce_counts():
    bf = BruteForce(4)
    dos = bf.energy_dos()
    assert sum(dos.values()) == 2 ** 16
    # two ground states E = -2N, and no state with E = -2N + 4 (one flipped
    # spin costs 8): levels are spaced by 4, the first excitation is at +8
    assert dos[-32] == 2
    assert -28 not in dos
    assert dos[-24] == 2 * 16
    assert all((e + 32) % 4 == 0 for e in dos)


def test_transfer_matrix_dos_equals_enumeration_L4():
    assert transfer_matrix_dos(4) == BruteForce(4).energy_dos()


def test_transfer_matrix_dos_low_energy_counts_L6():
    """Counts fixed by hand: from the two ground states (E = -2N) a flipped
    cluster costs 2 per broken bond. One spin breaks 4 bonds, an adjacent
    pair 6 (2N pairs); 8 broken bonds come from two non-adjacent spins
    (N(N-1)/2 - 2N), straight (2N) and bent (4N) triples and 2 x 2 squares
    (N). Flipping every spin of one sublattice maps E to -E, and the
    level spacing is 4."""
    g = transfer_matrix_dos(6)
    N = 36
    assert sum(g.values()) == 2 ** N
    assert g[-2 * N] == 2
    assert -2 * N + 4 not in g
    assert g[-2 * N + 8] == 2 * N
    assert g[-2 * N + 12] == 2 * 2 * N
    assert g[-2 * N + 16] == 2 * (N * (N - 1) // 2 - 2 * N + 2 * N + 4 * N + N)
    assert all(g[e] == g[-e] for e in g)
    assert all((e + 2 * N) % 4 == 0 for e in g)


@pytest.mark.parametrize("L", [4, 6])
@pytest.mark.parametrize("beta", [0.1, 0.3, BETA_C, 0.7, 1.2])
def test_transfer_matrix_dos_lnZ_vs_kaufman(L, beta):
    g = transfer_matrix_dos(L)
    lw = np.array([math.log(c) - beta * e for e, c in g.items()])
    m = lw.max()
    lnZ = m + math.log(float(np.exp(lw - m).sum()))
    assert lnZ == pytest.approx(kaufman_lnZ(L, beta), rel=1e-12)


def test_beta_zero_values():
    bf = BruteForce(4)
    a = bf.averages(0.0)
    assert a["betaF_per_N"] == pytest.approx(-math.log(2.0), abs=1e-15)
    assert a["S_per_N"] == pytest.approx(math.log(2.0), abs=1e-15)
    assert a["e"] == pytest.approx(0.0, abs=1e-15)
    # <M^2> = N at beta = 0 (independent spins) -> m2 = 1/N
    assert a["m2"] == pytest.approx(1.0 / 16, rel=1e-13)
    assert kaufman_lnZ(64, 0.0) == 64 * 64 * math.log(2.0)


def test_kaufman_derivatives_match_bruteforce():
    bf = BruteForce(4)
    for beta in [0.1, 0.4, 0.9]:
        k = kaufman_observables(4, beta)
        a = bf.averages(beta)
        assert k["e"] == pytest.approx(a["e"], abs=1e-7)
        assert k["C"] == pytest.approx(a["C"], abs=1e-5)


def test_kaufman_large_L_thermodynamic_limit():
    # Onsager: at beta_c the infinite-lattice energy is -sqrt(2); L = 128 is close
    e = kaufman_observables(128, BETA_C)["e"]
    assert abs(e + math.sqrt(2.0)) < 5e-3
    # deep in the ordered phase e -> -2
    assert kaufman_observables(64, 2.0)["e"] == pytest.approx(-2.0, abs=1e-5)
