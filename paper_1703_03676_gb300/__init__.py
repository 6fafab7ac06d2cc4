"""GB300 population-annealing engine for the 2D Ising model (arXiv:1703.03676).

Thin ctypes binding of the C ABI in include/pa.h. Every step of the method
runs in the CUDA kernels of ``csrc/``; this module only marshals arguments.
There is no CPU fallback: without the compiled library or a GPU the calls
raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

__all__ = ["PAConfig", "PARun", "PAError", "lib", "philox_device", "footprint_bytes",
           "SPIN_INT8", "SPIN_BITS32", "SPIN_MSC32", "SPIN_REPLICA8", "OBS_FIELDS"]

SPIN_INT8, SPIN_BITS32, SPIN_MSC32, SPIN_REPLICA8 = 0, 1, 2, 3
HIST_E, HIST_M, HIST_ESUM = 0, 1, 2

_STATUS = {0: "ok", 1: "done", 2: "again", -1: "invalid argument", -2: "out of memory", -3: "capacity",
           -4: "extinct", -5: "timeout", -6: "cuda error", -7: "invalid state", -8: "stalled"}


class PAError(RuntimeError):
    def __init__(self, status: int, where: str):
        detail = ""
        if status == -6 and _lib is not None:
            detail = " - " + (_lib.pa_last_error_message() or b"").decode(errors="replace")
        super().__init__(f"{where}: {_STATUS.get(status, status)} ({status}){detail}")
        self.status = status
        self.kind = _STATUS.get(status, str(status))


class _Config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("theta", ctypes.c_int32), ("R", ctypes.c_int64),
                ("beta0", ctypes.c_double), ("beta_f", ctypes.c_double), ("dbeta", ctypes.c_double),
                ("overlap", ctypes.c_double), ("seed", ctypes.c_uint64), ("spin_format", ctypes.c_int32),
                ("record_histograms", ctypes.c_int32), ("capacity", ctypes.c_int64),
                ("group_threads", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("potts_q", ctypes.c_int32), ("block_warps", ctypes.c_int32)]


class _TuneKey(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("spin_format", ctypes.c_int32), ("dim", ctypes.c_int32),
                ("potts_q", ctypes.c_int32), ("r_log2", ctypes.c_int32), ("batched", ctypes.c_int32),
                ("sms", ctypes.c_int32), ("gpu", ctypes.c_char * 64)]


class _TuneChoice(ctypes.Structure):
    _fields_ = [("group_threads", ctypes.c_int32), ("block_warps", ctypes.c_int32),
                ("attempts_per_ns", ctypes.c_double), ("candidates", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _Obs(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("e", ctypes.c_double), ("C", ctypes.c_double),
                ("abs_m", ctypes.c_double), ("m2", ctypes.c_double), ("m4", ctypes.c_double),
                ("betaF_per_N", ctypes.c_double), ("S_per_N", ctypes.c_double), ("lnQ", ctypes.c_double),
                ("R", ctypes.c_int64), ("families", ctypes.c_int64)]


class _StepInfo(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("delta", ctypes.c_double), ("S", ctypes.c_double),
                ("R", ctypes.c_int64), ("R_prev", ctypes.c_int64), ("kmin_prev", ctypes.c_int32),
                ("kmin", ctypes.c_int32), ("kmax", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("T4", ctypes.c_uint64), ("T8", ctypes.c_uint64), ("families", ctypes.c_int64)]


OBS_FIELDS = [f for f, _ in _Obs._fields_]
_OBS_DTYPE = np.dtype([(f, np.float64) for f in OBS_FIELDS[:9]] + [("R", np.int64), ("families", np.int64)])

_lib = None

# (name, restype, argtypes) of every exported symbol of include/pa.h
_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("pa_create", ctypes.c_int, [ctypes.POINTER(_Config), _P, ctypes.POINTER(_P)]),
    ("pa_step", ctypes.c_int, [_P]),
    ("pa_run", ctypes.c_int, [_P]),
    ("pa_sync", ctypes.c_int, [_P]),
    ("pa_launch", ctypes.c_int, [_P]),
    ("pa_reset", ctypes.c_int, [_P, ctypes.c_uint64]),
    ("pa_num_rows", ctypes.c_int, [_P, _I64P]),
    ("pa_observables", ctypes.c_int, [_P, ctypes.POINTER(_Obs), ctypes.c_int64, _I64P]),
    ("pa_step_info_get", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(_StepInfo)]),
    ("pa_histogram", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _I64P, ctypes.c_int64]),
    ("pa_population", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int8), ctypes.c_int64, _I64P]),
    ("pa_population_hash", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    ("pa_replicas", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _I64P,
                                   ctypes.c_int64, _I64P]),
    ("pa_mhr", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(_Obs)]),
    ("pa_ln_dos", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int64]),
    ("pa_mag_sums", ctypes.c_int, [_P, _P, ctypes.c_int64]),
    ("pa_phase_times", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), _I64P]),
    ("pa_kernel_launches", ctypes.c_int, [_P, _I64P]),
    ("pa_tune_key_of", ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_int32, ctypes.POINTER(_TuneKey)]),
    ("pa_autotune", ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_char_p, _P, ctypes.POINTER(_TuneChoice)]),
    ("pa_tune_cache_store", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_TuneKey), ctypes.POINTER(_TuneChoice)]),
    ("pa_tune_cache_lookup", ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_TuneKey), ctypes.POINTER(_TuneChoice),
                                            ctypes.POINTER(ctypes.c_int32)]),
    ("pa_launch_shape", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]),
    ("pa_footprint_bytes", ctypes.c_size_t, [ctypes.POINTER(_Config)]),
    ("pa_config_default", None, [ctypes.POINTER(_Config)]),
    ("pa_destroy", None, [_P]),
    ("pa_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("pa_last_error_message", ctypes.c_char_p, []),
    ("pa_philox_device", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_uint64, _P, _P]),
    ("pa_batch_create", ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    ("pa_batch_launch", ctypes.c_int, [_P]),
    ("pa_batch_sync", ctypes.c_int, [_P]),
    ("pa_batch_run", ctypes.c_int, [_P]),
    ("pa_batch_reset", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    ("pa_batch_get", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P)]),
    ("pa_batch_phase_times", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), _I64P]),
    ("pa_batch_shape", ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    ("pa_batch_destroy", None, [_P]),
    ("pa_step_async", ctypes.c_int, [_P]),
    ("pa_checkpoint", ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    ("pa_restore", ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    ("pa_create_couplings", ctypes.c_int, [ctypes.POINTER(_Config), _P, _P, _P, ctypes.POINTER(_P)]),
    ("pa_create_scheduled", ctypes.c_int, [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                           _P, ctypes.POINTER(_P)]),
    ("pa_weighted_average", ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _P]),
    ("pa_serve", ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
    ("pa_gather", ctypes.c_int, [_P, ctypes.c_int64, _P, ctypes.c_int64, ctypes.c_int32, _P, _P,
                                 ctypes.POINTER(ctypes.c_double)]),
    ("pa_measure_rng_peak", ctypes.c_int, [ctypes.c_int64, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    ("pa_measure_pipe_peak", ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    ("pa_selftest_bulk_wait", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
    ("pa_resample", ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int64, _P,
                                   ctypes.c_int64, _I64P, _P]),
    ("pa_resample_noalloc", ctypes.c_int, [_P, ctypes.c_int64, _P, _P, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_int64, _P, ctypes.c_int64, _I64P, _P]),
]


def lib() -> ctypes.CDLL:
    """The engine library, built for sm_103a on first use."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libpa_gb300.so is missing and could not be built")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, where: str, ok=(0,)):
    if st not in ok:
        raise PAError(st, where)
    return st


def _stream_handle(stream):
    """cudaStream_t for the engine. None: the context creates its own stream.
    torch's legacy default stream (handle 0) cannot be shared: pass a
    torch.cuda.Stream to order engine work with other work on it."""
    if stream is None:
        return ctypes.c_void_p(None)
    h = stream if isinstance(stream, int) else stream.cuda_stream
    if h == 0:
        raise ValueError("pass a torch.cuda.Stream (not the legacy default stream) or None")
    return ctypes.c_void_p(h)


@dataclass
class PAConfig:
    """Run parameters (see include/pa.h, pa_config)."""
    L: int = 16
    R: int = 1000
    theta: int = 10
    beta_f: float = 1.0
    dbeta: float = 0.01          # <= 0: adaptive steps
    overlap: float = 0.85
    seed: int = 1
    spin_format: int = SPIN_BITS32
    record_histograms: bool = False
    capacity: int = 0
    group_threads: int = 0
    use_graph: bool = True
    profile: bool = False
    dim: int = 2                 # 3: the L x L x L simple cubic lattice (bit-packed, L in 8..64)
    potts_q: int = 0             # 2..8: the q-state Potts model (SPIN_INT8, square lattice)
    block_warps: int = 0         # warps per CTA of warp-group sweeps (1, 2, 4, 8; 0: default/tuned)

    @property
    def n_sites(self) -> int:
        return self.L ** (3 if self.dim == 3 else 2)

    @property
    def nlev(self) -> int:
        """Entries of every histogram: energy levels k = (E + dim N)/4."""
        if self.potts_q:
            return 2 * self.n_sites + 1
        d = 3 if self.dim == 3 else 2
        return d * self.n_sites // 2 + 1

    def _c(self) -> _Config:
        c = _Config()
        c.L, c.theta, c.R = self.L, self.theta, self.R
        c.beta0, c.beta_f, c.dbeta, c.overlap = 0.0, self.beta_f, self.dbeta, self.overlap
        c.seed = self.seed & 0xFFFFFFFFFFFFFFFF
        c.spin_format = self.spin_format
        c.record_histograms = int(bool(self.record_histograms))
        c.capacity = self.capacity
        c.group_threads = self.group_threads
        c.use_graph = int(bool(self.use_graph))
        c.profile = int(bool(self.profile))
        c.dim = self.dim
        c.potts_q = self.potts_q
        c.block_warps = self.block_warps
        return c


def footprint_bytes(cfg: PAConfig) -> int:
    c = cfg._c()
    return int(lib().pa_footprint_bytes(ctypes.byref(c)))


class PARun:
    """One population-annealing run on the GPU (a pa_ctx)."""

    def __init__(self, cfg: PAConfig, stream=None, schedule=None, couplings=None):
        """schedule: optional increasing betas beta_1..beta_n to follow
        (pa_create_scheduled), e.g. the row betas of an adaptive first run.
        couplings: optional (Jr, Jd) int8 L x L arrays of +-1 (pa_create_couplings)."""
        self.cfg = cfg
        self._lib = lib()
        self._h = ctypes.c_void_p()
        c = cfg._c()
        if couplings is not None:
            assert schedule is None
            Jr = np.ascontiguousarray(couplings[0], dtype=np.int8).ravel()
            Jd = np.ascontiguousarray(couplings[1], dtype=np.int8).ravel()
            self._J = (Jr, Jd)
            _check(self._lib.pa_create_couplings(ctypes.byref(c), ctypes.c_void_p(Jr.ctypes.data),
                                                 ctypes.c_void_p(Jd.ctypes.data), _stream_handle(stream),
                                                 ctypes.byref(self._h)), "pa_create_couplings")
        elif schedule is None:
            _check(self._lib.pa_create(ctypes.byref(c), _stream_handle(stream), ctypes.byref(self._h)), "pa_create")
        else:
            b = np.ascontiguousarray(schedule, dtype=np.float64)
            _check(self._lib.pa_create_scheduled(ctypes.byref(c), b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 b.size, _stream_handle(stream), ctypes.byref(self._h)),
                   "pa_create_scheduled")
        self.N = cfg.n_sites

    # -- lifecycle
    def close(self):
        if self._h:
            self._lib.pa_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping
    def step(self) -> bool:
        """One temperature step; False once beta_f was already reached."""
        st = self._lib.pa_step(self._h)
        _check(st, "pa_step", ok=(0, 1))
        return st == 0

    def run(self):
        _check(self._lib.pa_run(self._h), "pa_run")
        return self

    def step_async(self) -> int:
        """Non-blocking step: 0 enqueued, 1 done, 2 previous step still running."""
        st = self._lib.pa_step_async(self._h)
        _check(st, "pa_step_async", ok=(0, 1, 2))
        return st

    def launch(self):
        """Enqueue the rest of the schedule without waiting."""
        _check(self._lib.pa_launch(self._h), "pa_launch")
        return self

    def reset(self, seed: int):
        """Back to step 0 with a new seed, keeping allocations."""
        _check(self._lib.pa_reset(self._h, seed & 0xFFFFFFFFFFFFFFFF), "pa_reset")
        self.cfg.seed = seed
        return self

    def sync(self):
        _check(self._lib.pa_sync(self._h), "pa_sync")

    # -- results
    def num_rows(self) -> int:
        n = ctypes.c_int64()
        _check(self._lib.pa_num_rows(self._h, ctypes.byref(n)), "pa_num_rows")
        return n.value

    def rows(self) -> np.ndarray:
        """Observables per step as a structured array (fields OBS_FIELDS)."""
        n = self.num_rows()
        buf = (_Obs * max(n, 1))()
        got = ctypes.c_int64()
        _check(self._lib.pa_observables(self._h, buf, n, ctypes.byref(got)), "pa_observables")
        out = np.zeros(got.value, dtype=_OBS_DTYPE)
        for i in range(got.value):
            for f in OBS_FIELDS:
                out[f][i] = getattr(buf[i], f)
        return out

    def step_info(self, step: int) -> dict:
        s = _StepInfo()
        _check(self._lib.pa_step_info_get(self._h, step, ctypes.byref(s)), "pa_step_info_get")
        return {f: getattr(s, f) for f, _ in _StepInfo._fields_ if f != "pad"}

    def histogram(self, step: int, kind: int = HIST_E) -> np.ndarray:
        out = np.zeros(self.cfg.nlev, dtype=np.int64)
        _check(self._lib.pa_histogram(self._h, step, kind, out.ctypes.data_as(_I64P), out.size), "pa_histogram")
        return out

    def population(self) -> np.ndarray:
        """Current population as int8 +1/-1 of shape (R_i, L, L)."""
        n = self.num_rows()
        R = self.step_info(n - 1)["R"]
        out = np.zeros((R,) + (self.cfg.L,) * (3 if self.cfg.dim == 3 else 2), dtype=np.int8)
        got = ctypes.c_int64()
        _check(self._lib.pa_population(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), R,
                                       ctypes.byref(got)), "pa_population")
        return out[: got.value]

    def population_hash(self) -> int:
        """FNV-1a 64 of the current population (pa_population_hash)."""
        h = ctypes.c_uint64()
        _check(self._lib.pa_population_hash(self._h, ctypes.byref(h)), "pa_population_hash")
        return h.value

    def replicas(self):
        """(E, M, family) of the current population."""
        n = self.num_rows()
        R = self.step_info(n - 1)["R"]
        E = np.zeros(R, dtype=np.int32)
        M = np.zeros(R, dtype=np.int32)
        F = np.zeros(R, dtype=np.int64)
        got = ctypes.c_int64()
        _check(self._lib.pa_replicas(self._h, E.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     M.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), F.ctypes.data_as(_I64P),
                                     R, ctypes.byref(got)), "pa_replicas")
        return E[: got.value], M[: got.value], F[: got.value]

    def ln_dos(self) -> np.ndarray:
        out = np.zeros(self.cfg.nlev, dtype=np.float64)
        _check(self._lib.pa_ln_dos(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size),
               "pa_ln_dos")
        return out

    def checkpoint(self) -> bytes:
        """Snapshot of the run at the current step boundary (pa_checkpoint)."""
        n = ctypes.c_size_t()
        _check(self._lib.pa_checkpoint(self._h, None, 0, ctypes.byref(n)), "pa_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.pa_checkpoint(self._h, buf, n.value, ctypes.byref(n)), "pa_checkpoint")
        return buf.raw[: n.value]

    def restore(self, blob: bytes):
        """Resume from a checkpoint of a run with the same configuration."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.pa_restore(self._h, buf, len(blob)), "pa_restore")
        return self

    def mag_sums(self) -> np.ndarray:
        """Per-level sums (N+1, 5) uint64: |M|, M^2 lo/hi, M^4 lo/hi."""
        out = np.zeros(self.cfg.nlev * 5, dtype=np.uint64)
        _check(self._lib.pa_mag_sums(self._h, ctypes.c_void_p(out.ctypes.data), out.size), "pa_mag_sums")
        return out.reshape(self.cfg.nlev, 5)

    def mhr(self, betas) -> np.ndarray:
        b = np.ascontiguousarray(betas, dtype=np.float64)
        buf = (_Obs * max(b.size, 1))()
        _check(self._lib.pa_mhr(self._h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), b.size, buf), "pa_mhr")
        out = np.zeros(b.size, dtype=_OBS_DTYPE)
        for i in range(b.size):
            for f in OBS_FIELDS:
                out[f][i] = getattr(buf[i], f)
        return out

    def phase_times(self):
        ms = (ctypes.c_double * 7)()
        n = (ctypes.c_int64 * 7)()
        _check(self._lib.pa_phase_times(self._h, ms, n), "pa_phase_times")
        names = ["tables", "counts", "scan", "parent", "sweep", "stats", "init"]
        return {k: (ms[i], n[i]) for i, k in enumerate(names)}

    def kernel_launches(self) -> int:
        """Kernels of the engine launched for this run so far (pa_kernel_launches)."""
        n = ctypes.c_int64()
        _check(self._lib.pa_kernel_launches(self._h, ctypes.byref(n)), "pa_kernel_launches")
        return n.value

    def launch_shape(self):
        g, b, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.pa_launch_shape(self._h, ctypes.byref(g), ctypes.byref(b), ctypes.byref(n)),
               "pa_launch_shape")
        return {"group_threads": g.value, "block_threads": b.value, "grid_blocks": n.value}


class _Request(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("cfg", _Config)]


class _RequestResult(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("attempts", ctypes.c_double),
                ("steps", ctypes.c_int64), ("footprint", ctypes.c_int64), ("status", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class _ServeOptions(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_active", ctypes.c_int32), ("keep", ctypes.c_int32),
                ("time_scale", ctypes.c_double), ("max_bypass", ctypes.c_int32), ("pad", ctypes.c_int32)]


def serve(requests, hbm_budget: int = 0, max_active: int = 8, time_scale: float = 1.0, keep: bool = False,
          max_bypass: int = 8):
    """Run the native request loop (pa_serve) on [(arrival_s, PAConfig)]
    sorted by arrival. A request that does not fit the budget may be passed
    by up to max_bypass later ones (0: strict arrival order). Returns
    (results, runs): results is a list of dicts (admit_s, finish_s,
    attempts, steps, footprint, status); runs holds the finished runs as
    PARun objects when keep is set."""
    n = len(requests)
    reqs = (_Request * max(n, 1))()
    for i, (t, c) in enumerate(requests):
        reqs[i].arrival_s = float(t)
        reqs[i].cfg = c._c()
    res = (_RequestResult * max(n, 1))()
    ctxs = (_P * max(n, 1))()
    opt = _ServeOptions(int(hbm_budget), int(max_active), int(bool(keep)), float(time_scale), int(max_bypass), 0)
    _check(lib().pa_serve(reqs, n, ctypes.byref(opt), res, ctxs if keep else None), "pa_serve")
    out = [{f: getattr(res[i], f) for f, _ in _RequestResult._fields_ if f != "pad"} for i in range(n)]
    runs = []
    if keep:
        for i, (t, c) in enumerate(requests):
            if ctxs[i]:
                r = PARun.__new__(PARun)
                r.cfg, r._lib, r._h, r.N = c, lib(), ctypes.c_void_p(ctxs[i]), c.n_sites
                runs.append(r)
            else:
                runs.append(None)
    return out, runs


def served_trace(n: int = 500, rate: float = 20.0, seed: int = 999, stream=None):
    """The served-PA request trace: request q draws Philox4x32-10 (key =
    seed) at counter (0, q, 4, 0): the gap to the previous arrival is
    -ln(1 - w0 2^-32)/rate seconds, L = {32, 64, 128, 256, 512}[w1 mod 5],
    R = 10000 + w2 mod 90001 (uniform in 10^4..10^5); seed 1000 + q.
    Returns [(arrival_s, L, R, seed)]. Uses the engine's device Philox."""
    import math

    import torch
    ctr = torch.zeros((n, 4), dtype=torch.int32)
    ctr[:, 1] = torch.arange(n, dtype=torch.int32)
    ctr[:, 2] = 4
    w = philox_device(ctr.cuda(), seed, stream).cpu().numpy().view(np.uint32).astype(np.int64)
    t = 0.0
    out = []
    for q in range(n):
        t += -math.log(1.0 - float(w[q, 0]) / 4294967296.0) / rate
        out.append((t, [32, 64, 128, 256, 512][w[q, 1] % 5], 10000 + int(w[q, 2] % 90001), 1000 + q))
    return out


class _BorrowedRun(PARun):
    """A run owned by a PABatch: read-only access through the PARun methods."""

    def __init__(self, handle, cfg):  # noqa: D401 - no pa_create
        self.cfg = cfg
        self._lib = lib()
        self._h = handle
        self.N = cfg.n_sites

    def close(self):
        self._h = ctypes.c_void_p()


class PABatch:
    """Independent fixed-schedule runs stepped together in one CUDA graph
    (pa_batch_*). runs[i] gives read-only access to run i."""

    def __init__(self, cfgs, stream=None):
        self._lib = lib()
        self.cfgs = list(cfgs)
        arr = (_Config * len(self.cfgs))(*[c._c() for c in self.cfgs])
        self._h = ctypes.c_void_p()
        _check(self._lib.pa_batch_create(arr, len(self.cfgs), _stream_handle(stream), ctypes.byref(self._h)),
               "pa_batch_create")
        self.runs = []
        for i, c in enumerate(self.cfgs):
            h = ctypes.c_void_p()
            _check(self._lib.pa_batch_get(self._h, i, ctypes.byref(h)), "pa_batch_get")
            self.runs.append(_BorrowedRun(h, c))

    def launch(self):
        _check(self._lib.pa_batch_launch(self._h), "pa_batch_launch")
        return self

    def sync(self):
        _check(self._lib.pa_batch_sync(self._h), "pa_batch_sync")
        return self

    def run(self):
        _check(self._lib.pa_batch_run(self._h), "pa_batch_run")
        return self

    def reset(self, seeds):
        arr = (ctypes.c_uint64 * len(self.cfgs))(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
        _check(self._lib.pa_batch_reset(self._h, arr), "pa_batch_reset")
        for c, s in zip(self.cfgs, seeds):
            c.seed = int(s)
        return self

    def phase_times(self):
        ms = (ctypes.c_double * 7)()
        n = (ctypes.c_int64 * 7)()
        _check(self._lib.pa_batch_phase_times(self._h, ms, n), "pa_batch_phase_times")
        names = ["tables", "counts", "scan", "parent", "sweep", "stats", "init"]
        return {k: (ms[i], n[i]) for i, k in enumerate(names)}

    def shape(self, i):
        g, nb = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.pa_batch_shape(self._h, i, ctypes.byref(g), ctypes.byref(nb)), "pa_batch_shape")
        return {"group_threads": g.value, "sweep_blocks": nb.value}

    def close(self):
        if self._h:
            for r in self.runs:
                r.close()
            self._lib.pa_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox_device(ctr, seed: int, stream=None):
    """Philox4x32-10 on the GPU: ctr is a CUDA int32/uint32 tensor of shape
    (n, 4); returns a tensor of the same shape with the outputs."""
    import torch
    assert ctr.is_cuda and ctr.dtype in (torch.int32, torch.uint32) and ctr.is_contiguous()
    out = torch.empty_like(ctr)
    torch.cuda.current_stream().synchronize()
    _check(lib().pa_philox_device(ctypes.c_void_p(ctr.data_ptr()), ctr.numel() // 4, seed & 0xFFFFFFFFFFFFFFFF,
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "pa_philox_device")
    return out


def measure_rng_peak(blocks_per_thread: int = 4096, stream=None) -> float:
    """Philox4x32-10 words per ns of the whole device (generator alone)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(sms * 2048, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    out = ctypes.c_double()
    _check(lib().pa_measure_rng_peak(blocks_per_thread, ctypes.c_void_p(sink.data_ptr()), _stream_handle(stream),
                                     ctypes.byref(out)), "pa_measure_rng_peak")
    return out.value


def selftest_bulk_wait(nbytes: int, copy: bool, tries: int, stream=None) -> str:
    """Outcome of the bounded bulk-copy wait self-test (pa_selftest_bulk_wait):
    "ok" when the bytes landed and match, "timeout" when the wait ran out."""
    return _STATUS.get(lib().pa_selftest_bulk_wait(nbytes, 1 if copy else 0, tries, _stream_handle(stream)),
                       "unknown")


PIPE_WIDE_MUL, PIPE_LOP3, PIPE_IMAD = 0, 1, 2


def measure_pipe_peak(pipe: int, iters: int = 4096, stream=None) -> float:
    """Measured lane instructions per ns (Gop/s) of one integer instruction
    class over the whole device: PIPE_WIDE_MUL (32x32->64 product by a
    constant, halves XORed, as in a Philox round),
    PIPE_LOP3 (three-input logic) or PIPE_IMAD (32-bit multiply-add)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.empty(sms * 2048, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    out = ctypes.c_double()
    _check(lib().pa_measure_pipe_peak(pipe, iters, ctypes.c_void_p(sink.data_ptr()), _stream_handle(stream),
                                      ctypes.byref(out)), "pa_measure_pipe_peak")
    return out.value


def gather(src, parent, words: int, dst=None, stream=None):
    """Standalone replica copy (pa_gather): src is a CUDA int32 tensor of
    n_src * words words, parent a CUDA int32 tensor of old-slot indices.
    Returns (dst, device ms)."""
    import torch
    assert src.is_cuda and src.dtype == torch.int32 and src.is_contiguous() and src.numel() % words == 0
    assert parent.is_cuda and parent.dtype == torch.int32 and parent.is_contiguous()
    n_new = parent.numel()
    if dst is None:
        dst = torch.empty(n_new * words, dtype=torch.int32, device=src.device)
    assert dst.is_cuda and dst.dtype == torch.int32 and dst.numel() >= n_new * words
    torch.cuda.current_stream().synchronize()
    ms = ctypes.c_double()
    _check(lib().pa_gather(ctypes.c_void_p(src.data_ptr()), src.numel() // words, ctypes.c_void_p(parent.data_ptr()),
                           n_new, words, ctypes.c_void_p(dst.data_ptr()), _stream_handle(stream), ctypes.byref(ms)),
           "pa_gather")
    return dst, ms.value


TUNE_KEY_FIELDS = ["L", "spin_format", "dim", "potts_q", "r_log2", "batched", "sms", "gpu"]


def _tune_key(d: dict) -> _TuneKey:
    k = _TuneKey()
    for f in TUNE_KEY_FIELDS[:-1]:
        setattr(k, f, int(d[f]))
    k.gpu = d["gpu"].encode() if isinstance(d["gpu"], str) else d["gpu"]
    return k


def _choice_dict(c: _TuneChoice) -> dict:
    return {"group_threads": c.group_threads, "block_warps": c.block_warps,
            "attempts_per_ns": c.attempts_per_ns, "candidates": c.candidates}


def tune_key(cfg: PAConfig, batched: bool = False) -> dict:
    """The autotuner's key of runs like cfg on the current device."""
    k = _TuneKey()
    c = cfg._c()
    _check(lib().pa_tune_key_of(ctypes.byref(c), int(bool(batched)), ctypes.byref(k)), "pa_tune_key_of")
    return {f: (getattr(k, f).decode() if f == "gpu" else getattr(k, f)) for f in TUNE_KEY_FIELDS}


def autotune(cfg: PAConfig, cache_path=None, stream=None) -> dict:
    """Tune (or recall) the sweep's launch shape for runs like cfg
    (pa_autotune); later runs created with group_threads = block_warps = 0
    and the same key use the choice."""
    c = cfg._c()
    out = _TuneChoice()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(lib().pa_autotune(ctypes.byref(c), path, _stream_handle(stream), ctypes.byref(out)), "pa_autotune")
    return _choice_dict(out)


def tune_cache_store(path, key: dict, choice: dict):
    """Write one choice into a tuner cache file (host only)."""
    c = _TuneChoice(int(choice["group_threads"]), int(choice["block_warps"]), float(choice["attempts_per_ns"]), 0, 0)
    k = _tune_key(key)
    _check(lib().pa_tune_cache_store(os.fsencode(path), ctypes.byref(k), ctypes.byref(c)), "pa_tune_cache_store")


def tune_cache_lookup(path, key: dict):
    """The choice stored for key in a tuner cache file, or None (host only)."""
    k = _tune_key(key)
    c = _TuneChoice()
    found = ctypes.c_int32()
    _check(lib().pa_tune_cache_lookup(os.fsencode(path), ctypes.byref(k), ctypes.byref(c), ctypes.byref(found)),
           "pa_tune_cache_lookup")
    return _choice_dict(c) if found.value else None


RESAMPLE_NOALLOC_MAX_OLD = 262144


def resample(levels, F, U, seed: int, step: int, capacity: int, stream=None, parent=None, noalloc=False):
    """Nearest-integer resampling on the GPU (pa_resample). levels: CUDA int32
    tensor of old-slot energy levels; F: CUDA int32 tensor (uint32 bits) of
    floor(tau_hat) per level; U: CUDA int64 tensor of ceil(frac 2^32) per
    level. Returns (parent, R_i) with parent a CUDA int32 tensor of length R_i.
    `parent` may be a caller-provided CUDA int32 tensor of length capacity.
    noalloc=True calls pa_resample_noalloc, which allocates no device memory
    (its scratch is a static array of the library; at most
    RESAMPLE_NOALLOC_MAX_OLD old slots; calls must not overlap on the GPU)."""
    import torch
    assert levels.is_cuda and levels.dtype == torch.int32 and levels.is_contiguous()
    assert F.is_cuda and F.dtype == torch.int32 and U.is_cuda and U.dtype == torch.int64 and F.numel() == U.numel()
    if parent is None:
        parent = torch.empty(capacity, dtype=torch.int32, device=levels.device)
    assert parent.is_cuda and parent.dtype == torch.int32 and parent.numel() >= capacity
    n = ctypes.c_int64()
    torch.cuda.current_stream().synchronize()
    fn = lib().pa_resample_noalloc if noalloc else lib().pa_resample
    _check(fn(ctypes.c_void_p(levels.data_ptr()), levels.numel(), ctypes.c_void_p(F.data_ptr()),
                             ctypes.c_void_p(U.data_ptr()), F.numel(), seed & 0xFFFFFFFFFFFFFFFF, step,
                             ctypes.c_void_p(parent.data_ptr()), capacity, ctypes.byref(n), _stream_handle(stream)),
           "pa_resample_noalloc" if noalloc else "pa_resample")
    return parent[: n.value], n.value


def weighted_average(rows_list, N: int) -> np.ndarray:
    """Combine M runs' row arrays (PARun.rows(), same betas) with free-energy
    weights (pa_weighted_average, Eq. weighted-average)."""
    m = len(rows_list)
    n = len(rows_list[0])
    buf = (_Obs * (m * n))()
    for r, rows in enumerate(rows_list):
        assert len(rows) == n
        for i in range(n):
            o = buf[r * n + i]
            for f in OBS_FIELDS:
                setattr(o, f, rows[f][i].item())
    out = (_Obs * n)()
    _check(lib().pa_weighted_average(buf, m, n, N, out), "pa_weighted_average")
    res = np.zeros(n, dtype=_OBS_DTYPE)
    for i in range(n):
        for f in OBS_FIELDS:
            res[f][i] = getattr(out[i], f)
    return res


def batch_config4_draw(n: int = 64, seed: int = 99, stream=None):
    """(L, R, theta) of the batched-PA workload: run r draws Philox4x32-10
    (key = seed) at counter (0, r, 3, 0); L = {16, 32, 64, 128}[w0 mod 4],
    R = 2000 + w1 mod 48001 (uniform in 2000..50000), theta =
    {10, 50, 100}[w2 mod 3]. Evaluated with the engine's device Philox."""
    import torch
    ctr = torch.zeros((n, 4), dtype=torch.int32)
    ctr[:, 1] = torch.arange(n, dtype=torch.int32)
    ctr[:, 2] = 3
    w = philox_device(ctr.cuda(), seed, stream).cpu().numpy().view(np.uint32).astype(np.int64)
    return [([16, 32, 64, 128][w[r, 0] % 4], 2000 + int(w[r, 1] % 48001), [10, 50, 100][w[r, 2] % 3])
            for r in range(n)]
