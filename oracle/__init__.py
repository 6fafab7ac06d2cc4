"""Population-annealing oracle: a plain, slow, single-threaded CPU statement
of the method of Barash, Weigel, Borovsky, Janke and Shchur,
"GPU accelerated population annealing algorithm" (arXiv:1703.03676).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The GPU engine (``paper_1703_03676_gb300``) never imports it and
shares no code with it.

Modules
-------
pa_oracle_core.c : Philox4x32-10, initial spins, Metropolis sweeps (also
                   the multi-spin-coded LCG variant, the +-J model, the
                   simple cubic lattice and the q-state Potts model),
                   measurement and the resampling uniforms (natural layout).
pa_oracle.py     : the population-annealing step logic (Sec. 2.1-2.4).
exact_ising.py   : exact 2D Ising references that pin the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pa_oracle_core.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpa_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part with gcc (no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def core() -> ctypes.CDLL:
    """The loaded C core, built on first use."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i8p = ctypes.POINTER(ctypes.c_int8)
            lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.oracle_init.argtypes = [ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_uint64, i8p]
            lib.oracle_sweep.argtypes = [ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_uint64,
                                         ctypes.c_int64, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.c_uint64, i8p]
            lib.oracle_sweep_msc.argtypes = lib.oracle_sweep.argtypes
            lib.oracle_sweep_j.argtypes = [ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, i8p, i8p, i8p]
            lib.oracle_measure_j.argtypes = [ctypes.c_int, ctypes.c_int64, i8p, i8p, i8p, i64p, i64p]
            lib.oracle_measure.argtypes = [ctypes.c_int, ctypes.c_int64, i8p, i64p, i64p]
            lib.oracle_msc_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32]
            lib.oracle_msc_word.restype = ctypes.c_uint32
            lib.oracle_init_potts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_uint64, i8p]
            lib.oracle_sweep_potts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_uint64,
                                               ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), i8p]
            lib.oracle_measure_potts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, i8p, i64p, i64p]
            lib.oracle_init3.argtypes = lib.oracle_init.argtypes
            lib.oracle_sweep3.argtypes = [ctypes.c_int, ctypes.c_int64, i64p, ctypes.c_uint64, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, i8p]
            lib.oracle_measure3.argtypes = lib.oracle_measure.argtypes
            lib.oracle_resample_words.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, u32p]
            lib.oracle_philox_many.argtypes = [ctypes.c_int64, u32p, ctypes.c_uint64, u32p]
            for f in (lib.oracle_philox4x32_10, lib.oracle_init, lib.oracle_sweep, lib.oracle_sweep_msc,
                      lib.oracle_sweep_j, lib.oracle_measure_j, lib.oracle_init3, lib.oracle_sweep3,
                      lib.oracle_init_potts, lib.oracle_sweep_potts, lib.oracle_measure_potts,
                      lib.oracle_measure3, lib.oracle_measure, lib.oracle_resample_words, lib.oracle_philox_many):
                f.restype = None
            _lib = lib
    return _lib
