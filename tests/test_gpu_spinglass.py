"""The +-J model on the GPU (pa_create_couplings) against the oracle with
the same couplings, bit for bit, on every bit-packed geometry and the byte
format; all-plus couplings give the ferromagnet."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from oracle.pa_oracle import PopulationAnnealing, random_couplings  # noqa: E402
from tests._parity import assert_row_close, compare_step  # noqa: E402

B32, I8 = eng.SPIN_BITS32, eng.SPIN_INT8

CASES = [
    ("L8-bits", 8, 600, 3, 1.0, 0.1, B32),
    ("L16-bits", 16, 900, 3, 1.0, 0.1, B32),
    ("L32-bits", 32, 1200, 2, 0.6, 0.1, B32),
    ("L64-bits", 64, 500, 2, 0.4, 0.1, B32),
    ("L128-bits", 128, 120, 1, 0.3, 0.15, B32),
    ("L6-int8", 6, 400, 3, 1.0, 0.1, I8),
    ("L16-bits-adaptive", 16, 800, 3, 1.2, 0.0, B32),
]


@pytest.mark.parametrize("name,L,R,theta,beta_f,dbeta,fmt", CASES, ids=[c[0] for c in CASES])
def test_spin_glass_parity(name, L, R, theta, beta_f, dbeta, fmt):
    J = random_couplings(L, 1000 + L)
    seed = 55 + L
    pa = PopulationAnnealing(L, R, theta, beta_f=beta_f, dbeta=dbeta, seed=seed, couplings=J)
    pa.run()
    run = eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, beta_f=beta_f, dbeta=dbeta, seed=seed, spin_format=fmt,
                                 record_histograms=True), couplings=J)
    run.run()
    rows = run.rows()
    assert len(rows) == len(pa.rows)
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"{name} row {i}")
        compare_step(run, pa, i)
    np.testing.assert_array_equal(run.population(), pa.pop)
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(E, pa.E)
    run.close()


def test_all_plus_couplings_equal_ferromagnet():
    L = 32
    ones = (np.ones((L, L), np.int8), np.ones((L, L), np.int8))
    cfg = eng.PAConfig(L=L, R=1000, theta=3, beta_f=0.4, dbeta=0.1, seed=9)
    a = eng.PARun(cfg, couplings=ones)
    b = eng.PARun(eng.PAConfig(**cfg.__dict__))
    a.run()
    b.run()
    np.testing.assert_array_equal(a.rows(), b.rows())
    np.testing.assert_array_equal(a.population(), b.population())
    a.close()
    b.close()


def test_odd_number_of_negative_bonds_rejected():
    L = 8
    Jr, Jd = random_couplings(L, 3)
    Jd = Jd.copy()
    Jd[0, 0] = -Jd[0, 0]
    with pytest.raises(eng.PAError) as ei:
        eng.PARun(eng.PAConfig(L=L, R=100, theta=1, beta_f=0.1, dbeta=0.1), couplings=(Jr, Jd))
    assert ei.value.kind == "invalid argument"
