"""The q-state Potts model on the GPU (pa_config.potts_q, byte states):
every integer result bit-identical to the oracle's Potts mode and the FP64
rows within 1e-12 for several q, lattice sizes (including partial Philox
blocks), replica groupings, fixed and adaptive steps and reweighting;
configurations the Potts path does not support are rejected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from oracle.pa_oracle import PopulationAnnealing  # noqa: E402
from tests._parity import assert_row_close, compare_step, fnv1a64  # noqa: E402

CASES = [
    # name, L, R, theta, beta_f, dbeta, seed, q, group_threads (0: default)
    ("q3-L4", 4, 700, 3, 1.0, 0.1, 31, 3, 0),
    ("q4-L6-ragged", 6, 500, 2, 1.2, 0.2, 32, 4, 0),
    ("q3-L16", 16, 600, 2, 1.0, 0.1, 33, 3, 0),
    ("q2-L16", 16, 300, 2, 1.0, 0.1, 34, 2, 0),
    ("q8-L32", 32, 200, 1, 1.0, 0.25, 35, 8, 0),
    ("q5-L16-g4", 16, 123, 2, 0.8, 0.2, 36, 5, 4),
    ("q3-L8-g1", 8, 77, 2, 0.6, 0.2, 38, 3, 1),
    ("q3-R1", 8, 1, 2, 0.6, 0.3, 39, 3, 0),
]


def oracle(L, R, theta, beta_f, dbeta, seed, q):
    pa = PopulationAnnealing(L, R, theta, beta_f=beta_f, dbeta=dbeta, seed=seed, potts_q=q, record_hist=True)
    pa.run()
    return pa


def engine(L, R, theta, beta_f, dbeta, seed, q, gt=0):
    return eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, beta_f=beta_f, dbeta=dbeta, seed=seed,
                                  spin_format=eng.SPIN_INT8, record_histograms=True, group_threads=gt, potts_q=q))


def check(run, pa, name):
    rows = run.rows()
    assert len(rows) == len(pa.rows)
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"{name} row {i}")
        compare_step(run, pa, i)
    pop = run.population()
    np.testing.assert_array_equal(pop, pa.pop)
    assert run.population_hash() == fnv1a64(pa.pop)
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(E, pa.E)
    np.testing.assert_array_equal(M, pa.M)
    np.testing.assert_array_equal(fam, pa.fam)
    np.testing.assert_array_equal(run.histogram(0, 2), pa.Hsum)


@pytest.mark.parametrize("name,L,R,theta,beta_f,dbeta,seed,q,gt", CASES, ids=[c[0] for c in CASES])
def test_potts_run_parity(name, L, R, theta, beta_f, dbeta, seed, q, gt):
    pa = oracle(L, R, theta, beta_f, dbeta, seed, q)
    run = engine(L, R, theta, beta_f, dbeta, seed, q, gt)
    if gt:
        assert run.launch_shape()["group_threads"] == gt
    run.run()
    check(run, pa, name)
    run.close()


def test_potts_adaptive_and_reweighting():
    pa = oracle(8, 500, 2, 1.5, 0.0, 37, 3)
    run = engine(8, 500, 2, 1.5, 0.0, 37, 3)
    run.run()
    check(run, pa, "adaptive")
    _, lno = pa.ln_dos()
    got = run.ln_dos()
    fin = np.isfinite(lno)
    np.testing.assert_array_equal(np.isfinite(got), fin)
    np.testing.assert_allclose(got[fin], lno[fin], rtol=1e-12, atol=1e-12)
    run.close()


def test_potts_unsupported_configs_rejected():
    bad = [dict(spin_format=eng.SPIN_BITS32), dict(spin_format=eng.SPIN_MSC32), dict(potts_q=1),
           dict(potts_q=9), dict(dim=3, L=8)]
    for kw in bad:
        base = dict(L=8, R=10, theta=1, beta_f=0.1, dbeta=0.05, spin_format=eng.SPIN_INT8, potts_q=3)
        base.update(kw)
        with pytest.raises(eng.PAError) as ei:
            eng.PARun(eng.PAConfig(**base))
        assert ei.value.kind == "invalid argument", kw
