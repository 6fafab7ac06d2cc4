"""Checkpoint and resume (pa_checkpoint / pa_restore): a run stopped at a
step boundary and resumed in a new context continues bit for bit like the
uninterrupted run, for fixed and adaptive steps and every spin format."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402

CASES = [
    ("bits-fixed", dict(L=32, R=1500, theta=3, beta_f=0.5, dbeta=0.05, spin_format=eng.SPIN_BITS32)),
    ("bits-adaptive", dict(L=16, R=900, theta=3, beta_f=0.5, dbeta=0.0, spin_format=eng.SPIN_BITS32)),
    ("int8-fixed", dict(L=6, R=500, theta=2, beta_f=0.4, dbeta=0.1, spin_format=eng.SPIN_INT8)),
    ("msc-fixed", dict(L=16, R=700, theta=3, beta_f=0.3, dbeta=0.05, spin_format=eng.SPIN_MSC32)),
    ("replica-fixed", dict(L=8, R=300, theta=2, beta_f=0.3, dbeta=0.1, spin_format=eng.SPIN_REPLICA8)),
    ("cubic-fixed", dict(L=8, R=600, theta=2, beta_f=0.5, dbeta=0.1, spin_format=eng.SPIN_BITS32, dim=3)),
    ("cubic-adaptive", dict(L=8, R=400, theta=2, beta_f=0.4, dbeta=0.0, spin_format=eng.SPIN_BITS32, dim=3)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_resume_equals_uninterrupted(name, kw):
    cfg = eng.PAConfig(seed=77, record_histograms=True, **kw)
    ref = eng.PARun(eng.PAConfig(**cfg.__dict__))
    ref.run()
    a = eng.PARun(eng.PAConfig(**cfg.__dict__))
    for _ in range(3):
        assert a.step()
    blob = a.checkpoint()
    a.close()
    b = eng.PARun(eng.PAConfig(**{**cfg.__dict__, "seed": 1}))  # the checkpoint brings its seed
    b.restore(blob)
    b.run()
    np.testing.assert_array_equal(b.rows(), ref.rows())
    np.testing.assert_array_equal(b.population(), ref.population())
    np.testing.assert_array_equal(b.histogram(0, 2), ref.histogram(0, 2))
    np.testing.assert_array_equal(b.mag_sums(), ref.mag_sums())
    ref.close()
    b.close()


def test_restore_rejects_other_lattice_with_the_same_site_count():
    """L = 16 simple cubic and L = 64 square lattices both have N = 4096."""
    a = eng.PARun(eng.PAConfig(L=16, R=100, theta=1, beta_f=0.2, dbeta=0.1, seed=3, dim=3))
    assert a.step()
    blob = a.checkpoint()
    a.close()
    b = eng.PARun(eng.PAConfig(L=64, R=100, theta=1, beta_f=0.2, dbeta=0.1, seed=3))
    with pytest.raises(eng.PAError):
        b.restore(blob)
    b.close()


def test_restore_rejects_other_configuration():
    a = eng.PARun(eng.PAConfig(L=16, R=500, theta=2, beta_f=0.2, dbeta=0.1, seed=3))
    a.step()
    blob = a.checkpoint()
    b = eng.PARun(eng.PAConfig(L=16, R=501, theta=2, beta_f=0.2, dbeta=0.1, seed=3))
    with pytest.raises(eng.PAError):
        b.restore(blob)
    with pytest.raises(eng.PAError):
        b.restore(blob[:100])
    a.close()
    b.close()
