"""The simple cubic (L x L x L) Ising model on the GPU (pa_config.dim = 3,
bit-packed): every integer result bit-identical to the oracle's 3D mode and
the FP64 rows within 1e-12, for each lattice size and replica grouping
(warp groups, one replica per CTA), fixed and adaptive steps, reweighting;
configurations the 3D path does not support are rejected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from tests._parity import assert_row_close, compare_step, fnv1a64, oracle_run  # noqa: E402

B32 = eng.SPIN_BITS32

CASES = [
    # name, L, R, theta, beta_f, dbeta, seed, group_threads (0: default)
    ("L8", 8, 700, 3, 0.6, 0.1, 51, 0),
    ("L16", 16, 300, 2, 0.4, 0.1, 52, 0),
    ("L16-g16-ragged", 16, 150, 2, 0.3, 0.1, 53, 16),
    ("L16-g8", 16, 90, 1, 0.3, 0.15, 57, 8),
    ("L32-cta", 32, 40, 1, 0.3, 0.15, 54, 0),
    ("L32-warp", 32, 40, 1, 0.3, 0.15, 55, 32),
    ("L32-g16", 32, 21, 1, 0.2, 0.1, 58, 16),
    ("L64-cta", 64, 6, 1, 0.2, 0.1, 56, 0),
    ("R1", 8, 1, 2, 0.4, 0.2, 59, 0),
]


def engine_run(L, R, theta, beta_f, dbeta, seed, gt=0, **kw):
    return eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, beta_f=beta_f, dbeta=dbeta, seed=seed, spin_format=B32,
                                  record_histograms=True, group_threads=gt, dim=3, **kw))


@pytest.mark.parametrize("name,L,R,theta,beta_f,dbeta,seed,gt", CASES, ids=[c[0] for c in CASES])
def test_3d_run_parity(name, L, R, theta, beta_f, dbeta, seed, gt):
    pa = oracle_run(L, R, theta, beta_f, dbeta, seed, dim=3)
    pa.run()
    run = engine_run(L, R, theta, beta_f, dbeta, seed, gt)
    if gt:
        assert run.launch_shape()["group_threads"] == gt
    run.run()
    rows = run.rows()
    assert len(rows) == len(pa.rows)
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"{name} row {i}")
        compare_step(run, pa, i)
    pop = run.population()
    assert pop.shape == pa.pop.shape
    np.testing.assert_array_equal(pop, pa.pop)
    assert run.population_hash() == fnv1a64(pa.pop)
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(E, pa.E)
    np.testing.assert_array_equal(M, pa.M)
    np.testing.assert_array_equal(fam, pa.fam)
    np.testing.assert_array_equal(run.histogram(0, 2), pa.Hsum)
    run.close()


def test_3d_adaptive_and_reweighting():
    pa = oracle_run(8, 500, 2, 0.5, 0.0, 61, dim=3)
    pa.run()
    run = engine_run(8, 500, 2, 0.5, 0.0, 61)
    run.run()
    rows = run.rows()
    assert len(rows) == len(pa.rows)
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"adaptive row {i}")
        compare_step(run, pa, i)
    E_k, lno = pa.ln_dos()
    got = run.ln_dos()
    fin = np.isfinite(lno)
    np.testing.assert_array_equal(np.isfinite(got), fin)
    np.testing.assert_allclose(got[fin], lno[fin], rtol=1e-12, atol=1e-12)
    run.close()


def test_3d_unsupported_configs_rejected():
    bad = [dict(spin_format=eng.SPIN_INT8), dict(L=128), dict(L=12), dict(spin_format=eng.SPIN_MSC32),
           dict(group_threads=256, L=16), dict(dim=4)]
    for kw in bad:
        base = dict(L=16, R=10, theta=1, beta_f=0.1, dbeta=0.05, spin_format=B32, dim=3)
        base.update(kw)
        with pytest.raises(eng.PAError) as ei:
            eng.PARun(eng.PAConfig(**base))
        assert ei.value.kind == "invalid argument", kw
    with pytest.raises(eng.PAError):
        eng.PABatch([eng.PAConfig(L=16, R=10, theta=1, beta_f=0.1, dbeta=0.05, spin_format=B32, dim=3)])
