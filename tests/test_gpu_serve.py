"""Serving (pa_serve): requests admitted by arrival, concurrency limit and
HBM footprint, runs advanced without blocking (pa_step_async), finished
runs free their memory for the next. Each request's result must equal the
same configuration run alone, bit for bit, and the admission rule must
hold at every moment."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402

B32, I8 = eng.SPIN_BITS32, eng.SPIN_INT8


def requests():
    mix = [  # arrival (s), L, R, theta, dbeta (<= 0 adaptive), fmt
        (0.000, 32, 3000, 5, 0.0, B32),
        (0.001, 16, 1500, 5, 0.0, B32),
        (0.002, 64, 2000, 3, 0.0, B32),
        (0.004, 8, 800, 4, 0.05, B32),
        (0.010, 16, 2500, 5, 0.0, I8),
        (0.020, 128, 300, 2, 0.0, B32),
        (0.030, 32, 1000, 5, 0.02, B32),
        (0.050, 64, 1200, 2, 0.0, B32),
    ]
    out = []
    for q, (t, L, R, th, db, fmt) in enumerate(mix):
        out.append((t, eng.PAConfig(L=L, R=R, theta=th, beta_f=0.45, dbeta=db, overlap=0.85, seed=1000 + q,
                                    spin_format=fmt)))
    return out


def test_served_equals_alone_and_budget_holds():
    reqs = requests()
    fps = [eng.footprint_bytes(c) for _, c in reqs]
    budget = int(2.5 * max(fps))  # at most a few resident at once
    res, runs = eng.serve(reqs, hbm_budget=budget, max_active=4, keep=True, max_bypass=0)
    assert all(r["status"] == 0 for r in res), res
    # admission: in arrival order (no bypass), within budget and concurrency at all times
    admits = [r["admit_s"] for r in res]
    assert admits == sorted(admits)
    for i, (t, _) in enumerate(reqs):
        assert res[i]["admit_s"] >= t - 1e-6
    events = sorted([(r["admit_s"], 1, i) for i, r in enumerate(res)] + [(r["finish_s"], -1, i) for i, r in enumerate(res)],
                    key=lambda e: (e[0], e[1]))
    used, live = 0, 0
    for _, kind, i in events:
        if kind == 1:
            used += fps[i]
            live += 1
            assert live <= 4 and (used <= budget or live == 1)
        else:
            used -= fps[i]
            live -= 1
    # every request equals the same configuration run alone
    for (t, c), r in zip(reqs, runs):
        alone = eng.PARun(eng.PAConfig(**c.__dict__))
        alone.run()
        np.testing.assert_array_equal(r.rows(), alone.rows())
        np.testing.assert_array_equal(r.population(), alone.population())
        alone.close()
        r.close()
    assert sum(r["attempts"] for r in res) > 0


def test_step_async_equals_blocking_steps():
    c = eng.PAConfig(L=32, R=2000, theta=3, beta_f=0.4, dbeta=0.0, seed=77, spin_format=B32)
    a = eng.PARun(c)
    while True:
        st = a.step_async()
        if st == 1:
            break
    b = eng.PARun(eng.PAConfig(**c.__dict__))
    while b.step():
        pass
    np.testing.assert_array_equal(a.rows(), b.rows())
    a.close()
    b.close()


def test_trace_draw_matches_oracle_philox():
    from oracle.pa_oracle import philox_many
    got = eng.served_trace(12)
    ctr = np.zeros((12, 4), dtype=np.uint32)
    ctr[:, 1] = np.arange(12)
    ctr[:, 2] = 4
    w = philox_many(ctr, 999)
    t = 0.0
    for q in range(12):
        t += -math.log(1.0 - float(w[q, 0]) / 4294967296.0) / 20.0
        assert got[q] == (t, [32, 64, 128, 256, 512][int(w[q, 1]) % 5], 10000 + int(w[q, 2]) % 90001, 1000 + q)


def test_served_other_models_equal_alone():
    """Requests of the further models (simple cubic, q-state Potts, adaptive
    and fixed) served together with Ising ones: each equals its run alone."""
    cfgs = [
        eng.PAConfig(L=16, R=600, theta=3, beta_f=0.3, dbeta=0.0, seed=1101, spin_format=B32, dim=3),
        eng.PAConfig(L=16, R=900, theta=3, beta_f=0.8, dbeta=0.1, seed=1102, spin_format=I8, potts_q=3),
        eng.PAConfig(L=32, R=700, theta=3, beta_f=0.4, dbeta=0.0, seed=1103, spin_format=B32),
        eng.PAConfig(L=8, R=500, theta=2, beta_f=0.6, dbeta=0.0, seed=1104, spin_format=I8, potts_q=5),
        eng.PAConfig(L=32, R=200, theta=2, beta_f=0.3, dbeta=0.1, seed=1105, spin_format=B32, dim=3),
    ]
    reqs = [(0.001 * q, c) for q, c in enumerate(cfgs)]
    res, runs = eng.serve(reqs, hbm_budget=1 << 34, max_active=3, keep=True)
    assert all(r["status"] == 0 for r in res), res
    for (_, c), r in zip(reqs, runs):
        alone = eng.PARun(eng.PAConfig(**c.__dict__))
        alone.run()
        np.testing.assert_array_equal(r.rows(), alone.rows())
        np.testing.assert_array_equal(r.population(), alone.population())
        alone.close()
        r.close()


def test_large_request_passed_by_small_ones_then_admitted_alone():
    """A request larger than the whole budget is passed by at most max_bypass
    later small requests, then admitted once nothing else is resident and runs
    alone; every result equals its run alone."""
    def small(q):
        return eng.PAConfig(L=16, R=800, theta=3, beta_f=0.3, dbeta=0.05, seed=2000 + q, spin_format=B32)
    big = eng.PAConfig(L=128, R=3000, theta=2, beta_f=0.2, dbeta=0.05, seed=2100, spin_format=B32)
    reqs = [(0.0, small(0)), (0.0, big)] + [(0.0, small(q + 1)) for q in range(8)]
    fp_small, fp_big = eng.footprint_bytes(small(0)), eng.footprint_bytes(big)
    budget = 3 * fp_small
    assert fp_big > budget
    res, runs = eng.serve(reqs, hbm_budget=budget, max_active=3, keep=True, max_bypass=3)
    assert all(r["status"] == 0 for r in res), res
    big_admit, big_finish = res[1]["admit_s"], res[1]["finish_s"]
    passed = [q for q in range(2, len(reqs)) if res[q]["admit_s"] < big_admit]
    # every request has arrived at time 0: the first admission pass takes
    # requests 0, 2 and 3 (the big one does not fit next to 0); request 4
    # passes it too unless 0, 2 and 3 retire in the same pass of the loop, when
    # the big one finds the device empty first
    assert passed in ([2, 3], [2, 3, 4]), passed
    for q, r in enumerate(res):
        if q != 1:  # nothing else resident while the big run is
            assert r["finish_s"] <= big_admit + 1e-6 or r["admit_s"] >= big_finish - 1e-6, (q, r, res[1])
    for (_, c), r in zip(reqs, runs):
        alone = eng.PARun(eng.PAConfig(**c.__dict__))
        alone.run()
        np.testing.assert_array_equal(r.rows(), alone.rows())
        np.testing.assert_array_equal(r.population(), alone.population())
        alone.close()
        r.close()
