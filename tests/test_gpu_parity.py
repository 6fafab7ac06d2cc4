"""GPU engine vs the oracle, through the C ABI (include/pa.h).

Integer state (spins, energies, histograms, copy numbers through R_i,
family counts) must match bit for bit; the normaliser S and the adaptive
step size are compared bitwise too (both sides evaluate the same IEEE
operations in the same order); derived FP64 rows to 1e-12 relative.
Cases span several copy-count tiles with ragged tails, every bit-packed
lattice geometry (several rows per word, one word per row, several words
per row) and the byte format at odd row lengths.
"""
import math

import numpy as np
import pytest

from tests._parity import REL_TOL, assert_row_close, compare_step, fnv1a64, oracle_run

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402

I8, B32, RP = eng.SPIN_INT8, eng.SPIN_BITS32, eng.SPIN_REPLICA8


def engine_run(L, R, theta, beta_f, dbeta, seed, fmt, **kw):
    cfg = eng.PAConfig(L=L, R=R, theta=theta, beta_f=beta_f, dbeta=dbeta, seed=seed, spin_format=fmt,
                       record_histograms=True, **kw)
    return eng.PARun(cfg)


def test_philox_device_matches_oracle():
    from oracle.pa_oracle import philox_many
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for seed in [0, 1, 0xDEADBEEF12345678]:
        t = torch.from_numpy(ctr.view(np.int32)).cuda()
        got = eng.philox_device(t, seed).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, philox_many(ctr, seed))


CASES = [
    # name, L, R, theta, beta_f, dbeta, seed, fmt
    ("L4-int8", 4, 300, 3, 1.0, 0.1, 5, I8),
    ("L6-int8-partial-quads", 6, 500, 2, 0.5, 0.05, 6, I8),
    ("L8-bits-8rows-per-word", 8, 700, 3, 1.0, 0.05, 7, B32),
    ("L16-bits", 16, 1000, 4, 0.3, 0.03, 12, B32),
    ("L32-bits-2rows-per-word", 32, 1500, 3, 0.5, 0.05, 8, B32),
    ("L64-bits-ragged-tiles", 64, 2600, 2, 0.6, 0.1, 9, B32),
    ("L128-bits-2words-per-row", 128, 300, 2, 0.3, 0.1, 10, B32),
    ("L256-bits", 256, 64, 1, 0.5, 0.25, 13, B32),
    ("L512-bits", 512, 16, 1, 1.0, 0.5, 14, B32),
    ("L10-int8", 10, 1100, 2, 0.4, 0.1, 15, I8),
    ("L6-replica-parallel", 6, 700, 2, 0.4, 0.1, 17, RP),
    ("L16-replica-parallel-ragged", 16, 1300, 3, 0.3, 0.05, 18, RP),
    # degenerate populations: one replica (one level, tau = 1: resampling is
    # the identity) and two
    ("R1-bits", 16, 1, 3, 0.5, 0.1, 21, B32),
    ("R1-int8", 6, 1, 2, 0.4, 0.2, 23, I8),
    ("R2-bits", 8, 2, 2, 0.6, 0.2, 22, B32),
]

CTA_CASES = [
    # one replica per 256-thread CTA (CTA-wide barriers between colour phases)
    ("L128-cta", 128, 300, 2, 0.3, 0.1, 10),
    ("L256-cta", 256, 40, 1, 0.5, 0.25, 16),
]


@pytest.mark.parametrize("name,L,R,theta,beta_f,dbeta,seed,fmt", CASES, ids=[c[0] for c in CASES])
def test_run_parity(name, L, R, theta, beta_f, dbeta, seed, fmt):
    pa = oracle_run(L, R, theta, beta_f, dbeta, seed)
    pa.run()
    run = engine_run(L, R, theta, beta_f, dbeta, seed, fmt)
    run.run()
    rows = run.rows()
    assert len(rows) == len(pa.rows)
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"{name} row {i}")
        compare_step(run, pa, i)
    np.testing.assert_array_equal(run.population(), pa.pop)
    assert run.population_hash() == fnv1a64(pa.pop)
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(E, pa.E)
    np.testing.assert_array_equal(M, pa.M)
    np.testing.assert_array_equal(fam, pa.fam)
    np.testing.assert_array_equal(run.histogram(0, 2), pa.Hsum)
    run.close()


@pytest.mark.parametrize("name,L,R,theta,beta_f,dbeta,seed", CTA_CASES, ids=[c[0] for c in CTA_CASES])
def test_cta_group_parity(name, L, R, theta, beta_f, dbeta, seed):
    pa = oracle_run(L, R, theta, beta_f, dbeta, seed)
    pa.run()
    run = engine_run(L, R, theta, beta_f, dbeta, seed, B32, group_threads=256)
    assert run.launch_shape()["group_threads"] == 256
    run.run()
    rows = run.rows()
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"{name} row {i}")
        compare_step(run, pa, i)
    np.testing.assert_array_equal(run.population(), pa.pop)
    run.close()


@pytest.mark.parametrize("fmt", [I8, B32], ids=["int8", "bits"])
def test_config1_stepwise(fmt):
    """Plain PA, L=16, R=1000, theta=10, dbeta=0.01 to beta=1, seed 1: the
    population after every one of the 100 steps, bit for bit."""
    pa = oracle_run(16, 1000, 10, 1.0, 0.01, 1)
    run = engine_run(16, 1000, 10, 1.0, 0.01, 1, fmt)
    np.testing.assert_array_equal(run.population(), pa.pop)
    i = 0
    while run.step():
        pa.step()
        i += 1
        np.testing.assert_array_equal(run.population(), pa.pop, err_msg=f"step {i}")
        compare_step(run, pa, i)
    assert i == 100 and pa.done
    rows = run.rows()
    for j, ref in enumerate(pa.rows):
        assert_row_close(rows[j], ref, f"row {j}")
    run.close()


def test_int8_equals_bits_and_graph_equals_stepping():
    a = engine_run(32, 3000, 5, 1.0, 0.02, 21, I8)
    b = engine_run(32, 3000, 5, 1.0, 0.02, 21, B32, use_graph=True)
    c = engine_run(32, 3000, 5, 1.0, 0.02, 21, B32, use_graph=False, group_threads=4)
    a.run()
    b.run()
    c.run()
    ra, rb, rc = a.rows(), b.rows(), c.rows()
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(ra, rc)
    np.testing.assert_array_equal(a.population(), b.population())
    np.testing.assert_array_equal(a.population(), c.population())
    for r in (a, b, c):
        r.close()


@pytest.mark.parametrize("L,fmt", [(16, B32), (8, I8)])
def test_adaptive_parity(L, fmt):
    pa = oracle_run(L, 800, 5, 0.6, 0.0, 31, overlap=0.85)
    pa.run()
    run = engine_run(L, 800, 5, 0.6, 0.0, 31, fmt, overlap=0.85)
    run.run()
    rows = run.rows()
    assert len(rows) == len(pa.rows) > 3
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"adaptive row {i}")
        compare_step(run, pa, i)
    np.testing.assert_array_equal(run.population(), pa.pop)
    # multi-histogram reweighting (Eq. MHReq1)
    E_k, lno = pa.ln_dos()
    got = run.ln_dos()
    fin = np.isfinite(lno)
    np.testing.assert_array_equal(np.isfinite(got), fin)
    np.testing.assert_allclose(got[fin], lno[fin], rtol=1e-12, atol=1e-12)
    betas = [0.1, 0.3, 0.45, 0.6]
    m_ref = pa.mhr(betas)
    m_got = run.mhr(betas)
    # the engine's host loops evaluate Eq. MHReq1 in the oracle's order
    # (ascending levels, left-to-right sums, libm exp/log): same IEEE results
    for a, b in zip(m_got, m_ref):
        for f in ("e", "C", "betaF_per_N", "S_per_N", "abs_m", "m2", "m4"):
            x, y = float(a[f]), b[f]
            assert x == y or math.isclose(x, y, rel_tol=REL_TOL, abs_tol=1e-300), (f, x, y)
    # the exact integer sums behind the magnetisation reweighting
    ms = run.mag_sums()
    for k in range(L * L + 1):
        a, m2, m4 = pa.Msums[k]
        assert int(ms[k, 0]) == a
        assert int(ms[k, 1]) + (int(ms[k, 2]) << 64) == m2
        assert int(ms[k, 3]) + (int(ms[k, 4]) << 64) == m4
    run.close()


def test_capacity_failure_matches_oracle():
    from oracle.pa_oracle import OracleError
    pa = oracle_run(8, 500, 1, 1.0, 0.2, 3, capacity=500)
    with pytest.raises(OracleError):
        pa.run()
    bad = len(pa.records)  # steps completed before the failing one
    run = eng.PARun(eng.PAConfig(L=8, R=500, theta=1, beta_f=1.0, dbeta=0.2, seed=3, spin_format=B32,
                                 capacity=500, record_histograms=True))
    with pytest.raises(eng.PAError) as ei:
        run.run()
    assert ei.value.kind == "capacity"
    rows = run.rows()
    assert len(rows) == bad
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"row {i}")
    run.close()


def test_extinction_matches_oracle():
    """A population of two replicas that grew to more than two, with every
    expected copy number below one, dies out at the same step on both sides
    (L = 8, R = 2, seed 113: step 3); the rows before it agree."""
    from oracle.pa_oracle import OracleError
    pa = oracle_run(8, 2, 1, 1.0, 0.05, 113)
    with pytest.raises(OracleError) as oe:
        pa.run()
    assert oe.value.kind == "extinct"
    bad = len(pa.records)  # steps completed before the failing one
    for fmt in (B32, I8):
        run = eng.PARun(eng.PAConfig(L=8, R=2, theta=1, beta_f=1.0, dbeta=0.05, seed=113, spin_format=fmt,
                                     record_histograms=True))
        with pytest.raises(eng.PAError) as ei:
            run.run()
        assert ei.value.kind == "extinct"
        rows = run.rows()
        assert len(rows) == bad
        for i, ref in enumerate(pa.rows):
            assert_row_close(rows[i], ref, f"row {i}")
        run.close()


def test_invalid_configs_rejected():
    for kw in [dict(L=7), dict(L=24, spin_format=B32), dict(theta=0), dict(R=0), dict(beta_f=-1.0),
               dict(dbeta=0.0, overlap=1.5), dict(group_threads=3)]:
        base = dict(L=16, R=100, theta=1, beta_f=0.1, dbeta=0.05, spin_format=I8)
        base.update(kw)
        with pytest.raises(eng.PAError) as ei:
            eng.PARun(eng.PAConfig(**base))
        assert ei.value.kind == "invalid argument"


def test_schedule_reuse_and_weighted_average():
    """Sec. 2.3 / 2.2: run 1 adaptive, runs 2-3 follow its schedule with other
    seeds, then the free-energy-weighted average; every run and the
    combination match the oracle."""
    from oracle.pa_oracle import PopulationAnnealing, weighted_average
    L, R, theta = 16, 900, 4
    p1 = oracle_run(L, R, theta, 0.5, 0.0, 61)
    p1.run()
    sched = [r.beta for r in p1.rows[1:]]
    r1 = engine_run(L, R, theta, 0.5, 0.0, 61, B32)
    r1.run()
    rows1 = r1.rows()
    np.testing.assert_array_equal(rows1["beta"][1:], np.array(sched))
    oracle_runs, engine_rows = [p1], [rows1]
    for seed in (62, 63):
        pm = PopulationAnnealing(L, R, theta, seed=seed, schedule=sched)
        pm.run()
        rm = eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, seed=seed, spin_format=B32, record_histograms=True),
                       schedule=sched)
        rm.run()
        rows = rm.rows()
        for i, ref in enumerate(pm.rows):
            assert_row_close(rows[i], ref, f"scheduled seed {seed} row {i}")
            compare_step(rm, pm, i)
        np.testing.assert_array_equal(rm.population(), pm.pop)
        oracle_runs.append(pm)
        engine_rows.append(rows)
        rm.close()
    comb = eng.weighted_average(engine_rows, L * L)
    ref = weighted_average([p.rows for p in oracle_runs])
    for i, g in enumerate(ref):
        for f in ("e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N"):
            x, y = float(comb[f][i]), g[f]
            assert x == y or math.isclose(x, y, rel_tol=REL_TOL, abs_tol=1e-300), (i, f, x, y)
    r1.close()
