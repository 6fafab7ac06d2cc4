"""Helpers shared by the GPU parity tests: run the oracle and the engine on
the same configuration and compare what must agree bit for bit."""
from __future__ import annotations

import math

import numpy as np

from oracle.pa_oracle import PopulationAnnealing

ROW_FIELDS = ["beta", "e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N", "lnQ"]
REL_TOL = 1e-12  # derived FP64 rows (integer parts are compared exactly)


def oracle_run(L, R, theta, beta_f, dbeta, seed, overlap=0.85, capacity=0, dim=2):
    pa = PopulationAnnealing(L, R, theta, beta_f=beta_f, dbeta=dbeta, seed=seed, overlap=overlap,
                             capacity=capacity, record_hist=True, dim=dim)
    return pa


def assert_row_close(got, ref, where=""):
    for f in ROW_FIELDS:
        a, b = float(got[f]), float(getattr(ref, f))
        if a == b:
            continue
        assert math.isclose(a, b, rel_tol=REL_TOL, abs_tol=1e-300), (where, f, a, b)
    assert int(got["R"]) == ref.R, (where, "R")
    assert int(got["families"]) == ref.families, (where, "families")


def compare_step(run, pa, i):
    """Integer state of step i must match exactly."""
    info = run.step_info(i)
    rec = pa.records[i]
    assert info["R"] == rec.R, (i, "R", info["R"], rec.R)
    assert info["families"] == rec.families, (i, "families")
    if i > 0:
        assert info["S"] == rec.S, (i, "S", info["S"], rec.S)  # bitwise: same IEEE ops in the same order
        assert info["delta"] == rec.delta, (i, "delta", info["delta"], rec.delta)
        assert info["beta"] == rec.beta, (i, "beta")
        assert info["T4"] == rec.T4 and info["T8"] == rec.T8, (i, "thresholds")
        assert info["kmin_prev"] == rec.kmin_prev, (i, "kmin_prev")
    np.testing.assert_array_equal(run.histogram(i, 0), rec.H_E, err_msg=f"H_E step {i}")
    hm = run.histogram(i, 1)  # nlev entries; magnetisation levels use the first N + 1
    np.testing.assert_array_equal(hm[: rec.H_M.size], rec.H_M, err_msg=f"H_M step {i}")
    assert not hm[rec.H_M.size:].any(), (i, "H_M beyond N")


def fnv1a64(pop) -> int:
    """FNV-1a 64 over int8 +1/-1 spins (the pa_population_hash definition)."""
    h = 0xCBF29CE484222325
    for v in pop.astype(np.int8).ravel().view(np.uint8).tolist():
        h ^= v
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h
