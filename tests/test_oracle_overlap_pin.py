"""Independent pins for the adaptive step of Sec. 2.3: the histogram overlap
alpha(delta) = (1/R_{i-1}) sum_k H[k] min(1, tau_hat_k(delta)) and the step
chosen from it.

Each check derives the value another way than the oracle's code does:

* two occupied levels k0, k0 + 1 with counts a, b and a step whose weight
  e^{-4 delta} is exactly 1/2 or 1/4: S = a + b w and the overlap
  (a min(1, R/S) + b min(1, R w/S)) / R_{i-1} are exact rationals here
  (fractions.Fraction), for R != R_{i-1} as well;
* with R = R_{i-1} the overlap is the shared area of the population's
  energy distribution and its reweighted copy, sum_k min(P_k, P'_k) with
  P' normalised by its own sum (no S, no tau_hat);
* a wide binomial histogram is nearly Gaussian with sigma_E = 4 sqrt(n)/2,
  for which the overlap is 2 Phi(-delta sigma_E / 2);
* for two levels and R = R_{i-1} = a + b the target overlap alpha* is
  reached at w* = a (alpha* n - a) / (b (n - alpha* n + a)), so the
  bisection must return delta* = -ln(w*)/4.

The last tests plant plausible mistakes in a copy of the overlap (R for
R_{i-1}, a dropped min, the wrong sign of the exponent, half the energy
between adjacent levels) and check that the pins above reject each one.
(Weights counted from level 0 instead of kmin are no mistake: the common
factor exp(-4 delta kmin) cancels in tau_hat.)
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.pa_oracle import choose_delta, level_weights, normaliser_S, overlap_alpha

K = 64  # highest energy level of an 8 x 8 lattice (levels 0..64)


def two_level(a, b, k0=10):
    H = np.zeros(K + 1, dtype=np.int64)
    H[k0], H[k0 + 1] = a, b
    return H, k0, k0 + 1


def exact_two_level_alpha(a, b, R, R_prev, w: Fraction) -> Fraction:
    S = a + b * w
    return (a * min(Fraction(1), Fraction(R) / S) + b * min(Fraction(1), R * w / S)) / R_prev


# (a, b, R, R_prev, delta with exp(-4 delta) exact): both min branches occur
TWO_LEVEL_CASES = [
    (30, 70, 100, 100, math.log(2.0) / 4, Fraction(1, 2)),
    (30, 70, 100, 120, math.log(2.0) / 4, Fraction(1, 2)),
    (30, 70, 100, 80, math.log(4.0) / 4, Fraction(1, 4)),
    (500, 20, 480, 520, math.log(2.0) / 4, Fraction(1, 2)),
    (7, 993, 1000, 1000, math.log(4.0) / 4, Fraction(1, 4)),
    (250, 250, 600, 500, math.log(2.0) / 4, Fraction(1, 2)),
]


def pin_two_level(alpha_fn):
    """Largest relative deviation of alpha_fn from the exact rational value."""
    worst = 0.0
    for a, b, R, R_prev, delta, w in TWO_LEVEL_CASES:
        assert math.exp(-4.0 * delta) == float(w)  # the step's weight is exact
        H, kmin, kmax = two_level(a, b)
        got = alpha_fn(H, kmin, kmax, R, R_prev, delta, K)
        ref = float(exact_two_level_alpha(a, b, R, R_prev, w))
        worst = max(worst, abs(got - ref) / ref)
    return worst


def shared_area(H, kmin, kmax, delta):
    """sum_k min(P_k, P'_k): P the histogram normalised to 1, P' the same
    histogram reweighted by exp(-4 delta k) and normalised to 1."""
    k = np.arange(H.size, dtype=np.float64)
    P = H / H.sum()
    Wt = H * np.exp(-4.0 * delta * (k - kmin))
    Pp = Wt / Wt.sum()
    return float(np.minimum(P, Pp).sum())


def random_histogram(seed):
    rng = np.random.default_rng(seed)
    H = np.zeros(K + 1, dtype=np.int64)
    lo = int(rng.integers(0, 30))
    width = int(rng.integers(5, 30))
    H[lo:lo + width] = rng.integers(0, 200, width)
    H[lo] = max(H[lo], 1)
    H[lo + width - 1] = max(H[lo + width - 1], 1)
    return H, lo, lo + width - 1


def pin_shared_area(alpha_fn):
    worst = 0.0
    for seed in range(12):
        H, kmin, kmax = random_histogram(seed)
        R = int(H.sum())
        for delta in (0.0, 0.003, 0.02, 0.1, 0.4):
            got = alpha_fn(H, kmin, kmax, R, R, delta, K)
            worst = max(worst, abs(got - shared_area(H, kmin, kmax, delta)))
    return worst


def binomial_histogram(n=40000, total=10 ** 7):
    from scipy.stats import binom
    k = np.arange(n + 1)
    H = np.round(binom.pmf(k, n, 0.5) * total).astype(np.int64)
    occ = np.nonzero(H)[0]
    return H, int(occ[0]), int(occ[-1]), n


def pin_gaussian(alpha_fn):
    from scipy.stats import norm
    H, kmin, kmax, n = binomial_histogram()
    R = int(H.sum())
    sigma_E = 4.0 * math.sqrt(n) / 2.0
    worst = 0.0
    for x in (0.1, 0.2, 0.38, 0.8):
        got = alpha_fn(H, kmin, kmax, R, R, x / sigma_E, n)
        worst = max(worst, abs(got - 2.0 * norm.cdf(-x / 2.0)))
    return worst


def test_overlap_two_level_exact():
    assert pin_two_level(overlap_alpha) < 4e-16


def test_overlap_equals_shared_area_of_distributions():
    assert pin_shared_area(overlap_alpha) < 1e-13


def test_overlap_gaussian_limit():
    pytest.importorskip("scipy")
    assert pin_gaussian(overlap_alpha) < 3e-5


@pytest.mark.parametrize("a,b,target", [(600, 400, 0.85), (300, 700, 0.9), (900, 100, 0.95), (50, 950, 0.85)])
def test_choose_delta_two_level_closed_form(a, b, target):
    n = a + b
    H, kmin, kmax = two_level(a, b)
    w_star = a * (target * n - a) / (b * (n - target * n + a))
    assert 0.0 < w_star < 1.0
    d_star = -math.log(w_star) / 4.0
    beta, beta_f = 0.2, 0.2 + 5.0 * d_star
    delta, final = choose_delta(H, kmin, kmax, n, n, beta, beta_f, target, K)
    assert not final
    assert delta == pytest.approx(d_star, rel=1e-12)
    # the remaining interval is taken whole when it already keeps the overlap
    beta_f2 = beta + 0.5 * d_star
    delta2, final2 = choose_delta(H, kmin, kmax, n, n, beta, beta_f2, target, K)
    assert final2 and delta2 == beta_f2 - beta


# ---- planted mistakes: every one must be caught by at least one pin
def _mutant(kind):
    def alpha(H, kmin, kmax, R, R_prev, delta, K_, estep=4):
        if kind == "wrong_sign":
            f = float(estep) * delta
            t = np.array([math.exp(f * float(d)) for d in range(kmax - kmin + 1)])
        elif kind == "half_energy_step":
            t = level_weights(delta, kmax - kmin + 1, estep // 2)
        else:
            t = level_weights(delta, kmax - kmin + 1, estep)
        S = normaliser_S(H, kmin, kmax, t, K_)
        acc = 0.0
        for k in range(kmin, kmax + 1):
            tau = (float(R) * float(t[k - kmin])) / S
            acc += float(H[k]) * (tau if kind == "no_min" else min(1.0, tau))
        return acc / float(R if kind == "R_for_R_prev" else R_prev)
    return alpha


@pytest.mark.parametrize("kind", ["R_for_R_prev", "no_min", "wrong_sign", "half_energy_step"])
def test_pins_reject_planted_mistakes(kind):
    bad = _mutant(kind)
    caught = pin_two_level(bad) > 1e-6 or pin_shared_area(bad) > 1e-6
    assert caught, kind


def test_mutant_harness_is_faithful():
    # the harness without a planted mistake passes every pin
    good = _mutant("none")
    assert pin_two_level(good) < 4e-16 and pin_shared_area(good) < 1e-13
