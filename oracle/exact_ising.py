"""Exact results for the 2D ferromagnetic Ising model on a periodic L x L torus.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this module; it
serves the tests, the golden-value script and ``__graft_entry__.smoke``.

These references pin the population-annealing oracle. The paper's model
(Sec. 3, Eq. hamiltonian) is H = -J sum_<ij> s_i s_j with J = 1 and periodic
boundaries; the paper notes (Sec. 3) that exact results exist for it and
uses beta_c = ln(1 + sqrt 2)/2. Four independent routes are given here:

* ``brute_force`` enumerates all 2^N states of a tiny lattice (N <= 20),
  also with +-J couplings (the disordered models the paper's method
  targets) and for the simple cubic 2 x 2 x 2 torus;
* ``transfer_matrix_lnZ`` evaluates Z = Tr T^L with the row-to-row transfer
  matrix (L <= 10);
* ``transfer_matrix_dos`` counts the exact integer density of states g(E)
  of tori up to 6 x 6 (2^36 states) with the same row transfer;
* ``kaufman_lnZ`` is Kaufman's (1949) closed form for the finite torus, in
  the four-product form also used by Beale (1996);
* ``potts_enumerate`` and ``potts_transfer_dos`` give the q-state Potts
  model's exact joint counts of (E, majority-state size) on tiny tori and
  its density of states for L = 4 (q = 2 is the Ising model with
  E_Potts = E_Ising / 2 - N, a pin between the two).

The tests check them against each other and against closed-form state
counts before any of them is used as a pin for the oracle.
"""
from __future__ import annotations

import math

import numpy as np

BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))


def _logsumexp(a: np.ndarray) -> float:
    m = float(np.max(a))
    return m + math.log(float(np.sum(np.exp(a - m))))


# ---------------------------------------------------------------- brute force
def enumerate_states_j(L: int, Jr, Jd):
    """E and M of all 2^N states of the +-J model: E = -sum_x,y (Jr s s_right
    + Jd s s_down)."""
    N = L * L
    if N > 20:
        raise ValueError("brute force limited to N <= 20")
    idx = np.arange(1 << N, dtype=np.int64)
    s = np.empty((1 << N, L, L), dtype=np.int32)
    for y in range(L):
        for x in range(L):
            s[:, y, x] = ((idx >> (y * L + x)) & 1) * 2 - 1
    Jr = np.asarray(Jr, dtype=np.int32)
    Jd = np.asarray(Jd, dtype=np.int32)
    E = -(Jr * s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (Jd * s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    return E.astype(np.int64), s.sum(axis=(1, 2)).astype(np.int64)


def enumerate_states3(L: int):
    """E and M of all 2^(L^3) states of the simple cubic L x L x L torus:
    E = -sum over every site's +x, +y and +z bond (for L = 2 the +x and -x
    neighbours coincide, so each such pair carries two bonds)."""
    N = L ** 3
    if N > 20:
        raise ValueError("brute force limited to N <= 20")
    idx = np.arange(1 << N, dtype=np.int64)
    s = np.empty((1 << N, L, L, L), dtype=np.int32)  # [state, z, y, x]
    for z in range(L):
        for y in range(L):
            for x in range(L):
                s[:, z, y, x] = ((idx >> ((z * L + y) * L + x)) & 1) * 2 - 1
    E = -(s * (np.roll(s, -1, axis=3) + np.roll(s, -1, axis=2) + np.roll(s, -1, axis=1))).sum(axis=(1, 2, 3))
    return E.astype(np.int64), s.sum(axis=(1, 2, 3)).astype(np.int64)


def enumerate_states(L: int):
    """Energy and magnetisation of every one of the 2^(L*L) configurations.

    Site (x, y) is bit y*L + x of the state index; bit set = spin +1.
    E = -sum over the 2N bonds (right and down neighbour of each site).
    """
    N = L * L
    if N > 20:
        raise ValueError("brute force limited to N <= 20")
    idx = np.arange(1 << N, dtype=np.int64)
    spins = np.empty((1 << N, L, L), dtype=np.int8)
    for y in range(L):
        for x in range(L):
            spins[:, y, x] = (((idx >> (y * L + x)) & 1) * 2 - 1).astype(np.int8)
    s = spins.astype(np.int32)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    M = s.sum(axis=(1, 2))
    return E.astype(np.int64), M.astype(np.int64)


class BruteForce:
    """Exact canonical averages of a tiny torus by full enumeration (square
    lattice, or simple cubic with dim = 3)."""

    def __init__(self, L: int, couplings=None, dim: int = 2):
        self.L = L
        self.N = L ** dim
        if dim == 3:
            E, M = enumerate_states3(L)
        else:
            E, M = enumerate_states(L) if couplings is None else enumerate_states_j(L, *couplings)
        # joint density of states g(E, M) as integer counts
        keys, counts = np.unique(np.stack([E, M], axis=1), axis=0, return_counts=True)
        self.E = keys[:, 0].astype(np.float64)
        self.M = keys[:, 1].astype(np.float64)
        self.g = counts.astype(np.float64)
        self.Ei = keys[:, 0]
        self.Mi = keys[:, 1]

    def energy_dos(self):
        """Exact g(E) as {E: count} (integers)."""
        out: dict[int, int] = {}
        for e, c in zip(self.Ei.tolist(), self.g.astype(np.int64).tolist()):
            out[e] = out.get(e, 0) + c
        return out

    def lnZ(self, beta: float) -> float:
        return _logsumexp(np.log(self.g) - beta * self.E)

    def boltzmann_energy_pmf(self, beta: float) -> dict[int, float]:
        """P(E) at inverse temperature beta."""
        lz = self.lnZ(beta)
        dos = self.energy_dos()
        return {e: math.exp(math.log(c) - beta * e - lz) for e, c in dos.items()}

    def averages(self, beta: float) -> dict[str, float]:
        """e, C, |m|, m^2, m^4, beta F / N and S / N at beta (Eq. observables,
        Eq. free-energy and Eq. entropy evaluated with exact weights)."""
        N = self.N
        lw = np.log(self.g) - beta * self.E
        lz = _logsumexp(lw)
        w = np.exp(lw - lz)
        e1 = float(np.sum(w * self.E))
        e2 = float(np.sum(w * self.E ** 2))
        am = float(np.sum(w * np.abs(self.M)))
        m2 = float(np.sum(w * self.M ** 2))
        m4 = float(np.sum(w * self.M ** 4))
        e = e1 / N
        betaF = -lz / N
        return {
            "e": e,
            "C": beta * beta * (e2 - e1 * e1) / N,
            "abs_m": am / N,
            "m2": m2 / N ** 2,
            "m4": m4 / N ** 4,
            "betaF_per_N": betaF,
            "S_per_N": beta * e - betaF,
        }


# ------------------------------------------------------------ transfer matrix
def transfer_matrix_lnZ(L: int, beta: float) -> float:
    """ln Z of the L x L torus as ln Tr T^L with the symmetric row transfer
    matrix T[a, b] = exp(beta/2 H_row(a)) exp(beta a.b) exp(beta/2 H_row(b)),
    where H_row(a) = sum_x a_x a_{x+1} (periodic) and a.b = sum_x a_x b_x."""
    if L > 10:
        raise ValueError("transfer matrix limited to L <= 10")
    n = 1 << L
    idx = np.arange(n)
    rows = np.array([[1 if (i >> x) & 1 else -1 for x in range(L)] for i in idx], dtype=np.float64)
    hrow = (rows * np.roll(rows, -1, axis=1)).sum(axis=1)
    inter = rows @ rows.T
    T = np.exp(0.5 * beta * hrow[:, None] + beta * inter + 0.5 * beta * hrow[None, :])
    lam = np.linalg.eigvalsh(T)
    lmax = float(np.max(np.abs(lam)))
    # Tr T^L = sum lam^L; L is even here or odd, both fine with signed powers
    ratio = lam / lmax
    s = float(np.sum(ratio ** L))
    return L * math.log(lmax) + math.log(s)


def transfer_matrix_dos(L: int) -> dict[int, int]:
    """Exact integer density of states g(E) of the L x L torus (L <= 6) by
    counting row sequences with the transfer matrix.

    Rows are states a in [0, 2^L) (bit x set = spin +1). Appending row b
    after row a adds dE(a, b) = -sum_x b_x b_{x+1} - sum_x a_x b_x. For every
    first row a0 the counts n[a0, b, E] of row sequences a0 .. b are carried
    row by row; closing the torus after L rows keeps b = a0. All counts stay
    below 2^(L*L) <= 2^36 < 2^53, so float64 matrix products are exact.
    """
    if not 2 <= L <= 6:
        raise ValueError("transfer-matrix density of states limited to 2 <= L <= 6")
    N = L * L
    n_rows = 1 << L
    idx = np.arange(n_rows)
    rows = np.array([[1 if (i >> x) & 1 else -1 for x in range(L)] for i in idx], dtype=np.int64)
    h = -(rows * np.roll(rows, -1, axis=1)).sum(axis=1)       # in-row bonds of b
    v = -(rows @ rows.T)                                      # bonds between rows a and b
    dE = v + h[None, :]                                       # [a, b]
    # energies in steps of 2 (dE is even); index i <-> E = 2 i - 2N
    n_e = 2 * N + 1
    cnt = np.zeros((n_rows, n_rows, n_e), dtype=np.float64)   # [a0, b, E index]
    cnt[idx, idx, N] = 1.0                                    # zero rows: E = 0
    for _ in range(L):
        nxt = np.zeros_like(cnt)
        by_e = cnt.transpose(0, 2, 1)                         # [a0, E index, b]
        for d in np.unique(dE):
            Md = (dE == d).astype(np.float64)                 # [b, b'] pairs adding energy d
            moved = (by_e @ Md).transpose(0, 2, 1)            # [a0, b', E index]
            shift = int(d) // 2
            if shift >= 0:
                nxt[:, :, shift:] += moved[:, :, :n_e - shift]
            else:
                nxt[:, :, :n_e + shift] += moved[:, :, -shift:]
        cnt = nxt
    # the L appended rows are rows 1..L; closing the torus needs row L == row 0
    closed = cnt[idx, idx, :].sum(axis=0)
    if float(closed.max()) >= 2.0 ** 53:
        raise ArithmeticError("count exceeds exact float64 range")
    out: dict[int, int] = {}
    for i in range(n_e):
        c = int(round(float(closed[i])))
        if c:
            out[2 * i - 2 * N] = c
    return out


# ------------------------------------------------------------ Kaufman (1949)
def _log_prod_2cosh(x: np.ndarray) -> float:
    # sum ln(2 cosh x) computed stably: ln(2cosh x) = |x| + ln(1 + e^{-2|x|})
    ax = np.abs(x)
    return float(np.sum(ax + np.log1p(np.exp(-2.0 * ax))))


def _log_abs_prod_2sinh(x: np.ndarray):
    """(ln |prod 2 sinh x|, sign of the product); sign 0 if a factor is 0."""
    if np.any(x == 0.0):
        return -math.inf, 0
    ax = np.abs(x)
    sign = int(np.prod(np.sign(x)))
    return float(np.sum(ax + np.log(-np.expm1(-2.0 * ax)))), sign


def kaufman_lnZ(L: int, beta: float) -> float:
    """ln Z of the L x L periodic square lattice (J = 1) from Kaufman's exact
    finite-size solution:

      Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4),  K = beta,
      Z1 = prod_{r=0}^{L-1} 2 cosh(L g_{2r+1}/2),  Z2 = prod 2 sinh(L g_{2r+1}/2),
      Z3 = prod_{r=0}^{L-1} 2 cosh(L g_{2r}/2),    Z4 = prod 2 sinh(L g_{2r}/2),
      cosh g_q = cosh 2K coth 2K - cos(q pi / L)   (q >= 1, g_q > 0),
      g_0 = 2K + ln tanh K                        (may be negative).
    """
    if beta <= 0.0:
        if beta == 0.0:
            return L * L * math.log(2.0)
        raise ValueError("beta must be >= 0")
    K = beta
    N = L * L
    c = math.cosh(2 * K) / math.tanh(2 * K)

    def gamma(q: np.ndarray) -> np.ndarray:
        g = np.arccosh(c - np.cos(q * math.pi / L))
        return g

    r = np.arange(L, dtype=np.float64)
    g_odd = gamma(2 * r + 1)
    g_even = gamma(2 * r)
    g_even[0] = 2 * K + math.log(math.tanh(K))
    a_odd = 0.5 * L * g_odd
    a_even = 0.5 * L * g_even
    terms = []  # (log|Zi|, sign)
    terms.append((_log_prod_2cosh(a_odd), 1))
    terms.append(_log_abs_prod_2sinh(a_odd))
    terms.append((_log_prod_2cosh(a_even), 1))
    terms.append(_log_abs_prod_2sinh(a_even))
    m = max(t[0] for t in terms if t[1] != 0)
    total = sum(t[1] * math.exp(t[0] - m) for t in terms if t[1] != 0)
    return math.log(0.5) + 0.5 * N * math.log(2.0 * math.sinh(2 * K)) + m + math.log(total)


def kaufman_observables(L: int, beta: float, h: float = 1e-4) -> dict[str, float]:
    """e, C, beta F/N and S/N from kaufman_lnZ by central differences in beta:
    e = -(1/N) d lnZ/d beta, C = (beta^2/N) d^2 lnZ/d beta^2."""
    N = L * L
    f0 = kaufman_lnZ(L, beta)
    if beta - 2 * h < 0:
        # one-sided near beta = 0 (only used for tiny beta in tests)
        fp, fpp = kaufman_lnZ(L, beta + h), kaufman_lnZ(L, beta + 2 * h)
        d1 = (-3 * f0 + 4 * fp - fpp) / (2 * h)
        d2 = (f0 - 2 * fp + fpp) / (h * h)
    else:
        fp, fm = kaufman_lnZ(L, beta + h), kaufman_lnZ(L, beta - h)
        d1 = (fp - fm) / (2 * h)
        d2 = (fp - 2 * f0 + fm) / (h * h)
    e = -d1 / N
    betaF = -f0 / N
    return {"e": e, "C": beta * beta * d2 / N, "betaF_per_N": betaF, "S_per_N": beta * e - betaF}


# ------------------------------------------------------------ q-state Potts
def potts_enumerate(L: int, q: int) -> dict[tuple[int, int], int]:
    """Exact counts of (E, M) over all q^N states of the L x L torus, with
    E = -(number of the 2N bonds joining equal states) and M the number of
    sites in the most populated state (q^N <= 2^22)."""
    N = L * L
    if q ** N > 1 << 22:
        raise ValueError("enumeration limited to q^N <= 2^22")
    idx = np.arange(q ** N, dtype=np.int64)
    s = np.empty((q ** N, L, L), dtype=np.int8)
    for y in range(L):
        for x in range(L):
            s[:, y, x] = (idx // q ** (y * L + x)) % q
    E = -((s == np.roll(s, -1, axis=2)).sum(axis=(1, 2)) + (s == np.roll(s, -1, axis=1)).sum(axis=(1, 2)))
    M = np.max(np.stack([(s == t).sum(axis=(1, 2)) for t in range(q)]), axis=0)
    keys, counts = np.unique(np.stack([E, M], axis=1), axis=0, return_counts=True)
    return {(int(e), int(m)): int(c) for (e, m), c in zip(keys, counts)}


def potts_averages(joint: dict, beta: float, N: int) -> dict[str, float]:
    """e, C, <M>/N, <M^2>/N^2, <M^4>/N^4, beta F/N, S/N from exact (E, M)
    counts (M: the majority state's size)."""
    E = np.array([k[0] for k in joint], dtype=np.float64)
    M = np.array([k[1] for k in joint], dtype=np.float64)
    lw = np.log(np.array(list(joint.values()), dtype=np.float64)) - beta * E
    lz = _logsumexp(lw)
    w = np.exp(lw - lz)
    e1, e2 = float(np.sum(w * E)), float(np.sum(w * E * E))
    betaF = -lz / N
    return {"e": e1 / N, "C": beta * beta * (e2 - e1 * e1) / N, "abs_m": float(np.sum(w * M)) / N,
            "m2": float(np.sum(w * M ** 2)) / N ** 2, "m4": float(np.sum(w * M ** 4)) / N ** 4,
            "betaF_per_N": betaF, "S_per_N": beta * e1 / N - betaF}


def potts_transfer_dos(L: int, q: int) -> dict[int, int]:
    """Exact g(E) of the q-state Potts model on the L x L torus by row
    transfer (q^L row states; counts below 2^53, so L = 4 for q <= 8)."""
    N = L * L
    if float(q) ** N >= 2.0 ** 53 or q ** L > 4096:
        raise ValueError("outside the exact float64 range")
    n_rows = q ** L
    idx = np.arange(n_rows)
    rows = np.array([[(i // q ** x) % q for x in range(L)] for i in idx], dtype=np.int64)
    h = -(rows == np.roll(rows, -1, axis=1)).sum(axis=1)                    # in-row bonds of b
    v = -(rows[:, None, :] == rows[None, :, :]).sum(axis=2)                 # bonds between rows a, b
    dE = v + h[None, :]                                                      # in [-2L, 0]
    n_e = 2 * N + 1                                                          # index i <-> E = -i
    cnt = np.zeros((n_rows, n_rows, n_e), dtype=np.float64)
    cnt[idx, idx, 0] = 1.0
    for _ in range(L):
        nxt = np.zeros_like(cnt)
        by_e = cnt.transpose(0, 2, 1)
        for d in np.unique(dE):
            moved = (by_e @ (dE == d).astype(np.float64)).transpose(0, 2, 1)
            shift = -int(d)                                                  # E decreases by |d|
            nxt[:, :, shift:] += moved[:, :, :n_e - shift]
        cnt = nxt
    closed = cnt[idx, idx, :].sum(axis=0)
    return {-i: int(round(float(closed[i]))) for i in range(n_e) if closed[i] > 0}
