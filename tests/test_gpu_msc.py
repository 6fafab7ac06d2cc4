"""The multi-spin-coded format (PA_SPIN_MSC32, Sec. 4 with the LCG variant)
against the oracle's multi-spin-coded mode, bit for bit: partial last
words (R not a multiple of 32), odd row lengths, adaptive steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from oracle.pa_oracle import PopulationAnnealing  # noqa: E402
from tests._parity import assert_row_close, compare_step  # noqa: E402

MSC = eng.SPIN_MSC32

CASES = [
    # name, L, R, theta, beta_f, dbeta, seed
    ("L4", 4, 100, 3, 1.0, 0.1, 5),
    ("L6-odd-rows", 6, 333, 2, 0.5, 0.05, 6),
    ("L16", 16, 1000, 4, 0.4, 0.05, 7),
    ("L32-ragged", 32, 1111, 3, 0.3, 0.1, 8),
    ("L64", 64, 700, 2, 0.2, 0.1, 9),
    ("L16-adaptive", 16, 800, 3, 0.5, 0.0, 10),
]


@pytest.mark.parametrize("name,L,R,theta,beta_f,dbeta,seed", CASES, ids=[c[0] for c in CASES])
def test_msc_parity(name, L, R, theta, beta_f, dbeta, seed):
    pa = PopulationAnnealing(L, R, theta, beta_f=beta_f, dbeta=dbeta, seed=seed, msc=True)
    pa.run()
    run = eng.PARun(eng.PAConfig(L=L, R=R, theta=theta, beta_f=beta_f, dbeta=dbeta, seed=seed, spin_format=MSC,
                                 record_histograms=True))
    run.run()
    rows = run.rows()
    assert len(rows) == len(pa.rows)
    for i, ref in enumerate(pa.rows):
        assert_row_close(rows[i], ref, f"{name} row {i}")
        compare_step(run, pa, i)
    np.testing.assert_array_equal(run.population(), pa.pop)
    E, M, fam = run.replicas()
    np.testing.assert_array_equal(E, pa.E)
    np.testing.assert_array_equal(fam, pa.fam)
    run.close()


def test_msc_step0_equals_single_spin_step0():
    """The initial spins do not depend on the coding."""
    a = eng.PARun(eng.PAConfig(L=16, R=500, theta=1, beta_f=0.1, dbeta=0.1, seed=3, spin_format=MSC))
    b = eng.PARun(eng.PAConfig(L=16, R=500, theta=1, beta_f=0.1, dbeta=0.1, seed=3, spin_format=eng.SPIN_BITS32))
    np.testing.assert_array_equal(a.population(), b.population())
    a.close()
    b.close()
