"""Population annealing for the Ising model (square lattice; also the simple
cubic one): the oracle's step logic.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The algorithm follows Sec. 2.1 of the paper (Machta's variant with unit
weights): start from R independent replicas at beta0 = 0; for each new
inverse temperature resample the population with the nearest-integer rule of
Eq. resampling-factors, run theta Metropolis sweeps per replica, and measure
the population averages of Eq. observables. The free energy follows
Eq. free-energy with Z_beta0 = 2^N, the entropy Eq. entropy. Sec. 2.3 gives
the adaptive step (histogram overlap alpha), Sec. 2.4 the multi-histogram
estimate of the density of states (Eq. MHReq1).

Readings where the paper is silent (each listed in the design notes):

* Energy level k = (E + 2N)/4 in [0, N]; magnetisation level m = (M + N)/2.
  On the simple cubic lattice (dim = 3) k = (E + 3N)/4 in [0, 3N/2], and a
  flip with all six neighbours aligned (dE = 12) needs x < ceil(exp(-12 beta)
  2^32).
* No sweeps at beta0: the random start is already in equilibrium there
  (Sec. 2.1); row 0 is emitted with ln Q_0 = 0.
* Fixed schedule: n = round((beta_f - beta0)/dbeta) steps with
  beta_i = beta0 + i*dbeta (a product, so no drift), step size dbeta in Q.
* Q is evaluated relative to the lowest occupied level kmin:
  S = sum_k H[k] t[k - kmin] with t[d] = exp(-(4 dbeta) d), summed as a fixed
  pairwise tree over the histogram padded with zeros to a power of two (the
  paper asks for a deterministic order, Sec. 3 "Resampling and
  measurements"); ln Q_i = ln S - ln R_{i-1} - dbeta * E_min, and
  tau_hat_k = R t[k - kmin] / S, equal to (R/R_{i-1}) tau_i of Sec. 2.1.
* Extra copy iff u < frac(tau_hat) with u = x 2^-32: as integers,
  x < U = ceil(frac * 2^32).
* Metropolis acceptance for dE = 4, 8: x < ceil(exp(-4 beta) 2^32),
  x < ceil(exp(-8 beta) 2^32); colour 0 is swept before colour 1.
* Population capacity R_cap = ceil(1.05 R) + 1024 unless set; a step that
  produces more replicas fails with "capacity", zero replicas with "extinct".
* Adaptive step: if alpha(beta_f - beta) >= alpha*, jump to beta_f;
  otherwise bisect [0, beta_f - beta] for 60 iterations keeping the lower end
  where alpha >= alpha*. alpha sums levels in ascending order.
* MHR includes row 0 (an exact beta = 0 sample) in the histogram sum.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import core


class OracleError(RuntimeError):
    """Raised with .kind in {"capacity", "extinct", "stalled"}."""

    def __init__(self, kind: str, msg: str):
        super().__init__(msg)
        self.kind = kind

    def __reduce__(self):
        # rebuilt from (kind, message) when it crosses a process boundary
        # (a worker of a multiprocessing pool raising it)
        return (OracleError, (self.kind, str(self)))


def _ptr(a: np.ndarray, ctype):
    import ctypes
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ------------------------------------------------------------- C-core wrappers
def philox4x32_10(ctr, key) -> tuple[int, int, int, int]:
    """Philox4x32-10 of one 128-bit counter (4 words) and 64-bit key (2 words)."""
    import ctypes
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    core().oracle_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def philox_many(ctr: np.ndarray, seed: int) -> np.ndarray:
    import ctypes
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    core().oracle_philox_many(ctr.shape[0], _ptr(ctr, ctypes.c_uint32), seed, _ptr(out, ctypes.c_uint32))
    return out


def init_spins(L: int, slots: np.ndarray, seed: int, dim: int = 2, potts_q: int = 0) -> np.ndarray:
    """Initial configurations: Ising spins +1/-1, or Potts states 0..q-1
    (potts_q >= 2, square lattice)."""
    import ctypes
    slots = np.ascontiguousarray(slots, dtype=np.int64)
    s = np.empty((slots.size,) + (L,) * dim, dtype=np.int8)
    if potts_q:
        core().oracle_init_potts(L, potts_q, slots.size, _ptr(slots, ctypes.c_int64), seed, _ptr(s, ctypes.c_int8))
        return s
    fn = core().oracle_init3 if dim == 3 else core().oracle_init
    fn(L, slots.size, _ptr(slots, ctypes.c_int64), seed, _ptr(s, ctypes.c_int8))
    return s


def sweep_potts(s: np.ndarray, slots: np.ndarray, seed: int, u0: int, theta: int, q: int, T) -> None:
    """theta Potts Metropolis sweeps in place; T = (T1, T2, T3, T4), the
    acceptance thresholds for dE = 1 .. 4."""
    import ctypes
    assert s.dtype == np.int8 and s.flags.c_contiguous
    slots = np.ascontiguousarray(slots, dtype=np.int64)
    t = (ctypes.c_uint64 * 4)(*[int(v) for v in T])
    core().oracle_sweep_potts(s.shape[1], q, slots.size, _ptr(slots, ctypes.c_int64), seed, u0, theta, t,
                              _ptr(s, ctypes.c_int8))


def measure_potts(s: np.ndarray, q: int) -> tuple[np.ndarray, np.ndarray]:
    """E = -(number of satisfied bonds) and M = size of the majority state."""
    import ctypes
    s = np.ascontiguousarray(s, dtype=np.int8)
    n = s.shape[0]
    E = np.empty(n, dtype=np.int64)
    M = np.empty(n, dtype=np.int64)
    core().oracle_measure_potts(s.shape[1], q, n, _ptr(s, ctypes.c_int8), _ptr(E, ctypes.c_int64),
                                _ptr(M, ctypes.c_int64))
    return E, M


def sweep(s: np.ndarray, slots: np.ndarray, seed: int, u0: int, theta: int, T4: int, T8: int,
          msc: bool = False, couplings=None, T12: int | None = None) -> None:
    """theta sweeps in place on s[r] (replica slot slots[r]); msc selects the
    multi-spin-coded random numbers (Philox-seeded LCG per 32 replicas);
    couplings = (Jr, Jd) int8 L x L arrays of the +-J model. A 3D population
    (s of shape (n, L, L, L)) needs T12 for flips with all six neighbours
    aligned."""
    import ctypes
    assert s.dtype == np.int8 and s.flags.c_contiguous
    slots = np.ascontiguousarray(slots, dtype=np.int64)
    L = s.shape[1]
    if s.ndim == 4:
        assert not msc and couplings is None and T12 is not None
        core().oracle_sweep3(L, slots.size, _ptr(slots, ctypes.c_int64), seed, u0, theta, T4, T8, T12,
                             _ptr(s, ctypes.c_int8))
        return
    if couplings is not None:
        assert not msc
        Jr = np.ascontiguousarray(couplings[0], dtype=np.int8)
        Jd = np.ascontiguousarray(couplings[1], dtype=np.int8)
        core().oracle_sweep_j(L, slots.size, _ptr(slots, ctypes.c_int64), seed, u0, theta, T4, T8,
                              _ptr(Jr, ctypes.c_int8), _ptr(Jd, ctypes.c_int8), _ptr(s, ctypes.c_int8))
        return
    fn = core().oracle_sweep_msc if msc else core().oracle_sweep
    fn(L, slots.size, _ptr(slots, ctypes.c_int64), seed, u0, theta, T4, T8, _ptr(s, ctypes.c_int8))


def measure(s: np.ndarray, couplings=None) -> tuple[np.ndarray, np.ndarray]:
    import ctypes
    s = np.ascontiguousarray(s, dtype=np.int8)
    n = s.shape[0]
    E = np.empty(n, dtype=np.int64)
    M = np.empty(n, dtype=np.int64)
    if s.ndim == 4:
        assert couplings is None
        core().oracle_measure3(s.shape[1], n, _ptr(s, ctypes.c_int8), _ptr(E, ctypes.c_int64),
                               _ptr(M, ctypes.c_int64))
        return E, M
    if couplings is not None:
        Jr = np.ascontiguousarray(couplings[0], dtype=np.int8)
        Jd = np.ascontiguousarray(couplings[1], dtype=np.int8)
        core().oracle_measure_j(s.shape[1], n, _ptr(s, ctypes.c_int8), _ptr(Jr, ctypes.c_int8),
                                _ptr(Jd, ctypes.c_int8), _ptr(E, ctypes.c_int64), _ptr(M, ctypes.c_int64))
        return E, M
    core().oracle_measure(s.shape[1], n, _ptr(s, ctypes.c_int8), _ptr(E, ctypes.c_int64),
                          _ptr(M, ctypes.c_int64))
    return E, M


def resample_words(seed: int, step: int, n: int) -> np.ndarray:
    import ctypes
    out = np.empty(n, dtype=np.uint32)
    core().oracle_resample_words(seed, step, n, _ptr(out, ctypes.c_uint32))
    return out


# ------------------------------------------------------------- scalar pieces
def metropolis_threshold(beta: float, dE: int) -> int:
    """ceil(exp(-beta dE) * 2^32): x < T accepts with probability exp(-beta dE)."""
    return int(math.ceil(math.ldexp(math.exp(-float(dE) * beta), 32)))


def pad_size(K: int) -> int:
    """Smallest power of two >= K + 1, the number of energy levels (K, the
    highest level, is N in 2D and 3N/2 in 3D)."""
    P = 1
    while P < K + 1:
        P *= 2
    return P


def pairwise_sum(a: np.ndarray) -> float:
    """Fixed binary tree: sum(a) = sum(left half) + sum(right half), len(a) a
    power of two. Computed level by level: neighbours are added in pairs."""
    a = np.asarray(a, dtype=np.float64)
    n = a.size
    assert n >= 1 and n & (n - 1) == 0
    while a.size > 1:
        a = a[0::2] + a[1::2]
    return float(a[0])


def level_weights(delta: float, ndiff: int, estep: int = 4) -> np.ndarray:
    """t[d] = exp(-(estep delta) d) for d = 0..ndiff-1 (libm exp, one call
    each); estep is the energy between levels (4 Ising, 1 Potts)."""
    f = float(estep) * delta
    return np.array([math.exp(-(f * float(d))) for d in range(ndiff)], dtype=np.float64)


def normaliser_S(H: np.ndarray, kmin: int, kmax: int, t: np.ndarray, K: int) -> float:
    """S = sum_k H[k] t[k - kmin] by the fixed pairwise tree (Eq. Q up to the
    factor exp(-dbeta E_min) / R_{i-1}); K is the highest energy level."""
    T = np.zeros(pad_size(K), dtype=np.float64)
    T[kmin:kmax + 1] = H[kmin:kmax + 1].astype(np.float64) * t[: kmax - kmin + 1]
    return pairwise_sum(T)


def copy_tables(R: int, t: np.ndarray, S: float):
    """tau_hat = R t / S; F = floor(tau_hat); U = ceil(frac(tau_hat) 2^32)."""
    tau = (float(R) * t) / S
    F = np.floor(tau)
    frac = tau - F
    U = np.ceil(frac * 4294967296.0)
    return tau, F.astype(np.int64), U.astype(np.int64)


def overlap_alpha(H: np.ndarray, kmin: int, kmax: int, R: int, R_prev: int, delta: float, K: int,
                  estep: int = 4) -> float:
    """Histogram overlap of Sec. 2.3: (1/R_{i-1}) sum_j min(1, tau_hat_j),
    evaluated over levels in ascending order (K: the highest energy level)."""
    t = level_weights(delta, kmax - kmin + 1, estep)
    S = normaliser_S(H, kmin, kmax, t, K)
    acc = 0.0
    for k in range(kmin, kmax + 1):
        acc += float(H[k]) * min(1.0, (float(R) * float(t[k - kmin])) / S)
    return acc / float(R_prev)


def choose_delta(H, kmin, kmax, R, R_prev, beta, beta_f, target, K, estep=4):
    """Adaptive step (Sec. 2.3): largest delta found by 60 bisection steps
    with alpha(delta) >= target; the whole remaining interval if it passes."""
    dmax = beta_f - beta
    if overlap_alpha(H, kmin, kmax, R, R_prev, dmax, K, estep) >= target:
        return dmax, True
    lo, hi = 0.0, dmax
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if overlap_alpha(H, kmin, kmax, R, R_prev, mid, K, estep) >= target:
            lo = mid
        else:
            hi = mid
    return lo, False


# ------------------------------------------------------------- the run
@dataclass
class StepRecord:
    step: int
    beta: float
    delta: float
    R: int                  # population after this step's resampling
    R_prev: int
    kmin_prev: int = 0      # lowest occupied level of the previous population
    S: float = 0.0
    lnQ: float = 0.0
    T4: int = 0
    T8: int = 0
    T12: int = 0                    # 3D only (six aligned neighbours)
    TP: tuple = ()                  # Potts only: thresholds for dE = 1 .. 4
    H_E: np.ndarray | None = None   # histogram of this step's population
    H_M: np.ndarray | None = None
    counts: np.ndarray | None = None  # r_j of the previous population
    families: int = 0
    sums: tuple = ()                # (sum E, sum E^2, sum |M|, sum M^2, sum M^4) as ints


@dataclass
class Row:
    beta: float
    e: float
    C: float
    abs_m: float
    m2: float
    m4: float
    betaF_per_N: float
    S_per_N: float
    lnQ: float
    R: int
    families: int

    N: int = 0

    def as_tuple(self):
        return (self.beta, self.e, self.C, self.abs_m, self.m2, self.m4,
                self.betaF_per_N, self.S_per_N, self.lnQ, self.R, self.families)


def moment_sums(E: np.ndarray, M: np.ndarray):
    """Exact integer population sums (Python ints, no overflow)."""
    Ei = [int(v) for v in E]
    Mi = [int(v) for v in M]
    return (sum(Ei), sum(v * v for v in Ei), sum(abs(v) for v in Mi),
            sum(v * v for v in Mi), sum(v ** 4 for v in Mi))


def make_row(beta: float, N: int, R: int, sums, sum_lnQ: float, lnQ: float, families: int,
             states: int = 2) -> Row:
    """Eq. observables, Eq. free-energy (Z_beta0 = states^N: 2 for Ising
    spins, q for the q-state Potts model) and Eq. entropy.
    C uses the exact integer numerator R sum E^2 - (sum E)^2, which equals
    beta^2 N (mean(e^2) - mean(e)^2) without cancellation."""
    sE, sE2, sAM, sM2, sM4 = sums
    fR, fN = float(R), float(N)
    e = float(sE) / (fR * fN)
    C = beta * beta * float(R * sE2 - sE * sE) / (fR * fR * fN)
    abs_m = float(sAM) / (fR * fN)
    m2 = float(sM2) / (fR * fN * fN)
    m4 = float(sM4) / (fR * fN * fN * fN * fN)
    betaF = -(fN * math.log(float(states)) + sum_lnQ) / fN
    return Row(beta, e, C, abs_m, m2, m4, betaF, beta * e - betaF, lnQ, R, families, N)


class PopulationAnnealing:
    """One PA run of the Ising model, step by step (Sec. 2.1): the square
    lattice (dim = 2, Sec. 3) or the simple cubic one (dim = 3). Energy
    levels are k = (E + dim N)/4 = 0 .. dim N/2."""

    def __init__(self, L: int, R: int, theta: int, beta_f: float = 1.0, dbeta: float = 0.01,
                 seed: int = 1, beta0: float = 0.0, overlap: float = 0.85,
                 capacity: int = 0, record_hist: bool = True, schedule=None, msc: bool = False,
                 couplings=None, dim: int = 2, potts_q: int = 0, workers: int = 1):
        """workers > 1 splits the population into that many contiguous
        blocks of replicas for the initial spins, the sweeps and the
        measurements, each block run by the same single-threaded C routine on
        its own thread. Replicas are independent given their slot numbers, so
        every result is identical to workers = 1."""
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        if potts_q and not (2 <= potts_q <= 8 and dim == 2 and not msc and couplings is None):
            raise ValueError("the Potts model: 2 <= q <= 8, square lattice, plain Philox sweeps")
        if L % 2 or L < (4 if dim == 2 and not potts_q else 2):
            raise ValueError("L must be even and >= 4 (>= 2 in 3D and for the Potts model)")
        if dim == 3 and (msc or couplings is not None):
            raise ValueError("the 3D model has plain Philox sweeps and J = 1")
        if beta0 != 0.0:
            raise ValueError("beta0 must be 0 (Z_beta0 = 2^N is known only there)")
        if R < 1 or theta < 1 or not (beta_f > beta0):
            raise ValueError("bad R, theta or beta_f")
        self.dim = dim
        self.q = int(potts_q)             # 0: Ising
        self.L, self.N, self.R, self.theta = L, L ** dim, int(R), int(theta)
        self.estep = 1 if self.q else 4   # energy between adjacent levels
        self.eoff = dim * self.N          # E_k = estep k - eoff
        # energy levels: Ising (E + dim N)/4 = 0 .. dim N/2; Potts E + 2N = 0 .. 2N
        self.nl = (2 * self.N if self.q else dim * self.N // 2) + 1
        self.seed = int(seed)
        self.beta_f = float(beta_f)
        self.dbeta = float(dbeta)
        # a given schedule beta_1 < ... < beta_n (Sec. 2.3: with M runs the
        # adaptive schedule of the first run is reused); step i then uses
        # delta_i = beta_i - beta_{i-1}
        self.schedule = None if schedule is None else [float(b) for b in schedule]
        self.adaptive = not (self.dbeta > 0.0) and self.schedule is None
        self.overlap = float(overlap)
        # default capacity ceil(1.05 R) + 1024 holds R_i = R +- O(sqrt R)
        self.R_cap = int(capacity) if capacity > 0 else int(math.ceil(self.R * 1.05)) + 1024
        if self.schedule is not None:
            self.n_fixed = len(self.schedule)
        else:
            self.n_fixed = int(math.floor((self.beta_f - beta0) / self.dbeta + 0.5)) if not self.adaptive else None
        self.record_hist = record_hist
        self.msc = bool(msc)  # multi-spin-coded sweeps (Sec. 4, LCG variant)
        # +-J couplings (Jr, Jd) shared by every replica; None: ferromagnet.
        # Levels k = (E + 2N)/4 need an even number of negative bonds.
        self.J = None
        if couplings is not None:
            Jr, Jd = (np.ascontiguousarray(a, dtype=np.int8).reshape(L, L) for a in couplings)
            if int((Jr < 0).sum() + (Jd < 0).sum()) % 2:
                raise ValueError("the number of negative couplings must be even")
            self.J = (Jr, Jd)
        self.step_index = 0
        self.beta = 0.0
        self.done = False
        self.partial = False
        self.workers = max(1, int(workers))
        # step 0: random configurations at beta0 = 0, measured, no sweeps
        slots = np.arange(self.R, dtype=np.int64)
        self.pop = self._blocks(lambda a, b: init_spins(L, slots[a:b], self.seed, dim, self.q), self.R,
                                combine=np.concatenate)
        self.E, self.M = self._measure(self.pop)
        self.fam = np.arange(self.R, dtype=np.int64)
        self.sum_lnQ = 0.0
        self.Hsum = np.zeros(self.nl, dtype=np.int64)
        # per energy level, summed over every measured replica of every step:
        # sum |M|, sum M^2, sum M^4 (Python ints, exact)
        self.Msums = [[0, 0, 0] for _ in range(self.nl)]
        self.records: list[StepRecord] = []
        self.rows: list[Row] = []
        self._measure_and_record(StepRecord(step=0, beta=0.0, delta=0.0, R=self.R, R_prev=self.R))

    # -- helpers
    def levels(self) -> np.ndarray:
        return (self.E + self.eoff) // self.estep

    def mlevels(self) -> np.ndarray:
        # Ising: number of up spins; Potts: M itself (the majority state's size)
        return self.M if self.q else (self.M + self.N) // 2

    def _blocks(self, fn, n, combine=None):
        """fn(a, b) on the replica blocks [a, b) of n replicas: one block, or
        `workers` contiguous blocks on a thread pool (the C routines release
        the interpreter lock). combine joins the blocks' results in order."""
        w = self.workers if n >= 2 * self.workers else 1
        cuts = [n * i // w for i in range(w + 1)]
        if w == 1:
            parts = [fn(0, n)]
        else:
            from concurrent.futures import ThreadPoolExecutor
            with ThreadPoolExecutor(w) as ex:
                parts = list(ex.map(lambda i: fn(cuts[i], cuts[i + 1]), range(w)))
        return combine(parts) if combine else None

    def _measure(self, s):
        def one(a, b):
            sub = s[a:b]
            return measure_potts(sub, self.q) if self.q else measure(sub, self.J)
        parts = self._blocks(one, s.shape[0], combine=list)
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])

    def _sweep(self, s, slots, u0, T4, T8, T12, TP):
        def one(a, b):  # s[a:b] is a contiguous block of s: swept in place
            if self.q:
                sweep_potts(s[a:b], slots[a:b], self.seed, u0, self.theta, self.q, TP)
            else:
                sweep(s[a:b], slots[a:b], self.seed, u0, self.theta, T4, T8, msc=self.msc, couplings=self.J,
                      T12=T12)
        self._blocks(one, s.shape[0])

    def _measure_and_record(self, rec: StepRecord):
        N = self.N
        H_E = np.bincount(self.levels(), minlength=self.nl).astype(np.int64)
        H_M = np.bincount(self.mlevels(), minlength=N + 1).astype(np.int64)
        self.Hsum += H_E
        for k, m in zip(self.levels().tolist(), self.M.tolist()):
            acc = self.Msums[k]
            acc[0] += abs(m)
            acc[1] += m * m
            acc[2] += m ** 4
        rec.families = int(np.unique(self.fam).size)
        rec.sums = moment_sums(self.E, self.M)
        if self.record_hist:
            rec.H_E, rec.H_M = H_E, H_M
        self.sum_lnQ += rec.lnQ
        self.records.append(rec)
        self.rows.append(make_row(rec.beta, N, rec.R, rec.sums, self.sum_lnQ, rec.lnQ, rec.families,
                                  self.q or 2))

    def n_steps_left(self):
        return None if self.adaptive else self.n_fixed - self.step_index

    # -- one temperature step (Sec. 2.1 steps 2-4)
    def step(self, sample: np.ndarray | None = None):
        """Advance one inverse-temperature step. With `sample` (new-slot
        indices, or a function of R_i returning them) only those replicas are
        swept and measured; the run then stops (used for full-size spot
        checks). Returns the record."""
        if self.done or self.partial:
            raise RuntimeError("run finished")
        N, R = self.N, self.R
        i = self.step_index + 1
        R_prev = self.E.size
        lv = self.levels()
        K = self.nl - 1
        H = np.bincount(lv, minlength=self.nl).astype(np.int64)
        occ = np.nonzero(H)[0]
        kmin, kmax = int(occ[0]), int(occ[-1])
        if self.schedule is not None:
            beta_new = self.schedule[i - 1]
            delta = beta_new - self.beta
            final = i == self.n_fixed
        elif self.adaptive:
            delta, final = choose_delta(H, kmin, kmax, R, R_prev, self.beta, self.beta_f, self.overlap, K,
                                        self.estep)
            if delta <= 0.0:
                raise OracleError("stalled", "adaptive step found no positive delta")
            beta_new = self.beta_f if final else self.beta + delta
        else:
            delta = self.dbeta
            beta_new = 0.0 + i * self.dbeta
            final = i == self.n_fixed
        # Eq. Q with the E_min shift, and the copy numbers of Eq. resampling-factors
        t = level_weights(delta, kmax - kmin + 1, self.estep)
        S = normaliser_S(H, kmin, kmax, t, K)
        _, F, U = copy_tables(R, t, S)
        x = resample_words(self.seed, i, R_prev).astype(np.int64)
        d = lv - kmin
        r = F[d] + (x < U[d]).astype(np.int64)
        R_new = int(r.sum())
        if R_new > self.R_cap:
            raise OracleError("capacity", f"R_{i} = {R_new} exceeds capacity {self.R_cap}")
        if R_new == 0:
            raise OracleError("extinct", f"population died out at step {i}")
        parent = np.repeat(np.arange(R_prev, dtype=np.int64), r)
        E_min = -self.eoff + self.estep * kmin
        lnQ = (math.log(S) - math.log(float(R_prev))) - delta * float(E_min)
        T4 = metropolis_threshold(beta_new, 4)
        T8 = metropolis_threshold(beta_new, 8)
        T12 = metropolis_threshold(beta_new, 12) if self.dim == 3 else None
        TP = tuple(metropolis_threshold(beta_new, d) for d in (1, 2, 3, 4)) if self.q else ()
        rec = StepRecord(step=i, beta=beta_new, delta=delta, R=R_new, R_prev=R_prev, kmin_prev=kmin,
                         S=S, lnQ=lnQ, T4=T4, T8=T8, T12=T12 or 0, TP=TP,
                         counts=r if self.record_hist else None)
        rec.parent = parent
        u0 = (i - 1) * self.theta
        if sample is not None:
            if callable(sample):
                sample = sample(R_new)
            sample = np.asarray(sample, dtype=np.int64)
            sub = np.ascontiguousarray(self.pop[parent[sample]])
            self._sweep(sub, sample, u0, T4, T8, T12, TP)
            rec.sample = sample
            rec.sample_pop = sub
            rec.sample_E, rec.sample_M = self._measure(sub)
            rec.sample_fam = self.fam[parent[sample]]
            self.partial = True
            self.records.append(rec)
            return rec
        self.pop = np.ascontiguousarray(self.pop[parent])
        self.fam = self.fam[parent]
        self._sweep(self.pop, np.arange(R_new, dtype=np.int64), u0, T4, T8, T12, TP)
        self.E, self.M = self._measure(self.pop)
        self.step_index = i
        self.beta = beta_new
        self.done = bool(final)
        self._measure_and_record(rec)
        return rec

    def run(self):
        while not self.done:
            self.step()
        return self.rows

    # -- multi-histogram reweighting (Sec. 2.4, Eq. MHReq1)
    # Plain loops in ascending level and row order, one libm exp/log per term
    # and sums accumulated left to right: every result is the value of the
    # formula evaluated in that stated order.
    def ln_dos(self) -> tuple[np.ndarray, np.ndarray]:
        """ln Omega(E_k) for every level with Hsum[k] > 0 (others -inf):
        ln Omega_k = ln Hsum_k - LSE_i(ln R_i + beta_i F_i - beta_i E_k),
        beta_i F_i = -(N ln 2 + sum_{l<=i} ln Q_l) (N ln q for Potts), with
        LSE_i(a_i) = m + ln sum_i exp(a_i - m), m = max_i a_i."""
        N = self.N
        E_k = [float(-self.eoff + self.estep * k) for k in range(self.nl)]
        betas = [r.beta for r in self.rows]
        lnR = [math.log(float(r.R)) for r in self.rows]
        bF = [r.betaF_per_N * N for r in self.rows]
        out = np.full(self.nl, -np.inf)
        for k in range(self.nl):
            if self.Hsum[k] > 0:
                a = [lnR[i] + bF[i] - betas[i] * E_k[k] for i in range(len(betas))]
                m = max(a)
                s = 0.0
                for v in a:
                    s += math.exp(v - m)
                out[k] = math.log(float(self.Hsum[k])) - (m + math.log(s))
        return np.array(E_k), out

    def mhr(self, betas) -> list[dict]:
        """Reweighted e, C, beta F / N, S / N and magnetisation moments at each
        beta: Z(beta) = sum_k Omega_k exp(-beta E_k), sums over the visited
        levels in ascending order (shifted by the largest exponent). The
        Boltzmann weight depends on E only, so the joint estimate
        Omega(E, M) of Eq. MHReq1 gives sum_M Omega(E, M) f(M) =
        Omega(E) * (sum of f(M) over every sample at level E) / Hsum(E)."""
        N = self.N
        fN = float(N)
        E_k, lno = self.ln_dos()
        lev = [k for k in range(self.nl) if np.isfinite(lno[k])]
        mic = {k: [float(self.Msums[k][j]) / float(self.Hsum[k]) for j in range(3)] for k in lev}
        out = []
        for b in betas:
            b = float(b)
            m = -math.inf
            for k in lev:
                m = max(m, lno[k] - b * E_k[k])
            Z = e1 = e2 = a1 = a2 = a4 = 0.0
            for k in lev:
                Ek = E_k[k]
                w = math.exp(lno[k] - b * Ek - m)
                Z += w
                e1 += w * Ek
                e2 += w * Ek * Ek
                a1 += w * mic[k][0]
                a2 += w * mic[k][1]
                a4 += w * mic[k][2]
            e1 /= Z
            e2 /= Z
            lnZ = m + math.log(Z)
            e = e1 / fN
            bF = -lnZ / fN
            out.append({"beta": b, "e": e, "C": b * b * (e2 - e1 * e1) / fN,
                        "betaF_per_N": bF, "S_per_N": b * e - bF, "lnZ": lnZ,
                        "abs_m": a1 / Z / fN, "m2": a2 / Z / (fN * fN), "m4": a4 / Z / (fN * fN * fN * fN)})
        return out


# ------------------------------------------------------------- M runs (Sec. 2.2)
def weighted_average(runs_rows):
    """Combine M independent runs with the same inverse temperatures
    (Eq. weighted-average). At each beta_i the weights are
    omega_m = exp(-beta_i F_m) / sum_m exp(-beta_i F_m), where
    -beta_i F_m = ln Z_m = -N (beta F / N)_m (Eq. free-energy). e, |m|, m^2
    and m^4 are averaged with these weights; C is formed from the weighted
    <e> and <e^2>, each run's <e^2> being C_m / (beta^2 N) + e_m^2 (at
    beta = 0 the C_m are averaged); the combined free energy is
    -beta F = ln((1/M) sum_m Z_m), and S/N = beta e - beta F / N.
    runs_rows: M lists of Row (same length, same betas)."""
    M = len(runs_rows)
    out = []
    for i in range(len(runs_rows[0])):
        rows = [rr[i] for rr in runs_rows]
        beta, N = rows[0].beta, rows[0].N
        for r in rows:
            if abs(r.beta - beta) > 1e-12 * max(1.0, abs(beta)) or r.N != N:
                raise ValueError("runs must share N and the inverse temperatures")
        lw = [-N * r.betaF_per_N for r in rows]
        top = max(lw)
        ex = [math.exp(x - top) for x in lw]
        Z = sum(ex)
        w = [x / Z for x in ex]
        e = sum(wi * r.e for wi, r in zip(w, rows))
        if beta > 0.0:
            e2 = sum(wi * (r.C / (beta * beta * N) + r.e * r.e) for wi, r in zip(w, rows))
            C = beta * beta * N * (e2 - e * e)
        else:
            C = sum(wi * r.C for wi, r in zip(w, rows))
        bF = -(top + math.log(Z) - math.log(M)) / N
        out.append({"beta": beta, "e": e, "C": C,
                    "abs_m": sum(wi * r.abs_m for wi, r in zip(w, rows)),
                    "m2": sum(wi * r.m2 for wi, r in zip(w, rows)),
                    "m4": sum(wi * r.m4 for wi, r in zip(w, rows)),
                    "betaF_per_N": bF, "S_per_N": beta * e - bF,
                    "R": sum(r.R for r in rows), "families": sum(r.families for r in rows), "weights": w})
    return out


def random_couplings(L: int, seed: int, p_negative: float = 0.5):
    """A +-J instance: (Jr, Jd) int8 L x L arrays, each bond -1 with
    probability p_negative (numpy's PCG64 from `seed`), with the last down
    bond flipped if needed so that the number of negative bonds is even."""
    rng = np.random.default_rng(seed)
    Jr = np.where(rng.random((L, L)) < p_negative, -1, 1).astype(np.int8)
    Jd = np.where(rng.random((L, L)) < p_negative, -1, 1).astype(np.int8)
    if int((Jr < 0).sum() + (Jd < 0).sum()) % 2:
        Jd[L - 1, L - 1] = -Jd[L - 1, L - 1]
    return Jr, Jd
