"""bench.py's host-side pieces without a GPU: the workload labels of the
default run and its labelled variants, and the oracle sample behind
cpu_baseline / --impl reference, which runs in spawned workers and so must
take the workload from its arguments, not from the module's globals, and
must finish when a population of its few replicas dies out."""
import pickle

import bench
from oracle.pa_oracle import OracleError

# L=8, R=2, theta=1, dbeta=0.05 to beta 1: with seed 113 the population dies
# out at step 2 (found by running the oracle; a population this small loses
# every replica when R_{i-1} > R and no copy number comes out above 0)
SMALL = dict(L=8, R=2, theta=1, beta_f=1.0, dbeta=0.05, dim=2, potts_q=0)
DYING_SEED = 113


def test_default_label_is_the_papers_run():
    assert bench.workload_label() == ("plain PA, 2D Ising L=64 periodic, R=20000, theta=100, beta 0->1 "
                                      "dbeta=0.005 (200 steps), bit-packed spins")


def test_variant_labels(monkeypatch):
    monkeypatch.setitem(bench.WL, "dim", 3)
    monkeypatch.setitem(bench.WL, "L", 16)
    assert "3D Ising (simple cubic) L=16^3" in bench.workload_label()
    assert bench.sites() == 4096
    monkeypatch.setitem(bench.WL, "dim", 2)
    monkeypatch.setitem(bench.WL, "potts_q", 3)
    monkeypatch.setitem(bench.WL, "dbeta", 0.0)
    label = bench.workload_label()
    assert "3-state Potts" in label and "adaptive" in label


def test_oracle_sample_uses_the_given_workload():
    base = dict(R=8, theta=2, beta_f=0.2, dbeta=0.1)
    for wl, n in ((dict(L=8, dim=2, potts_q=0), 64), (dict(L=4, dim=3, potts_q=0), 64),
                  (dict(L=8, dim=2, potts_q=3), 64)):
        att, secs, restarts = bench._oracle_sample((8, 1, 5, {**base, **wl}))
        # one step: N sites x theta sweeps x R_1 replicas (R_1 fluctuates around R)
        assert att % (n * 2) == 0 and att > 0 and secs >= 0 and restarts == 0


def test_oracle_error_survives_pickling():
    e = pickle.loads(pickle.dumps(OracleError("extinct", "population died out at step 3")))
    assert isinstance(e, OracleError) and e.kind == "extinct" and str(e) == "population died out at step 3"


def test_oracle_sample_restarts_a_population_that_died_out():
    att, secs, restarts = bench._oracle_sample((2, None, DYING_SEED, dict(SMALL)))
    assert restarts >= 1 and att > 0
    # a fixed number of steps is completed across the restarts
    att5, _, r5 = bench._oracle_sample((2, 5, DYING_SEED, dict(SMALL)))
    assert r5 >= 1 and att5 % (64 * 1) == 0 and att5 >= 5 * 64


def test_spawned_pool_finishes_when_a_population_dies_out(monkeypatch):
    for k, v in SMALL.items():
        monkeypatch.setitem(bench.WL, k, v)
    v, att, wall, restarts = bench.cpu_oracle(2, 2, None, DYING_SEED)
    assert restarts >= 1 and att > 0 and v > 0
    assert "died out" in bench.restart_note(restarts) and bench.restart_note(0) == ""


def test_cpu_baseline_object(monkeypatch):
    for k, v in SMALL.items():
        monkeypatch.setitem(bench.WL, k, v)
    obj = bench.cpu_baseline_obj(2, 2)
    assert obj["kind"] == "oracle" and obj["cores"] == 2 and obj["value"] > 0 and obj["unit"] == bench.UNIT
    assert "whole anneal" in obj["sample"]
