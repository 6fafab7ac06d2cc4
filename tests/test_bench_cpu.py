"""bench.py's host-side pieces without a GPU: the workload labels of the
default run and its labelled variants, and the oracle sample behind
cpu_baseline / --impl reference, which runs in spawned workers and so must
take the workload from its arguments, not from the module's globals."""
import bench


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
        att, secs = bench._oracle_sample((8, 1, 5, {**base, **wl}))
        # one step: N sites x theta sweeps x R_1 replicas (R_1 fluctuates around R)
        assert att % (n * 2) == 0 and att > 0 and secs >= 0
