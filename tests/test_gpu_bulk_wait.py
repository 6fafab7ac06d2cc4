"""The bounded wait behind the sweep's bulk prefetch: a barrier armed for
bytes that a copy delivers completes; one armed for bytes nothing delivers
gives up after its poll limit with a timeout status, and the context stays
usable (a run afterwards equals the oracle). No fault, trap or endless wait
is involved: the wait that runs out polls a bounded number of times."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from tests._parity import oracle_run  # noqa: E402


@pytest.mark.parametrize("nbytes", [16, 2048, 4096])
def test_copy_lands(nbytes):
    assert eng.selftest_bulk_wait(nbytes, True, 1 << 20) == "ok"


def test_wait_without_copy_times_out_and_context_stays_usable():
    assert eng.selftest_bulk_wait(2048, False, 2000) == "timeout"
    assert eng.selftest_bulk_wait(2048, True, 1 << 20) == "ok"
    r = eng.PARun(eng.PAConfig(L=128, R=40, theta=2, beta_f=0.1, dbeta=0.05, seed=77, spin_format=eng.SPIN_BITS32,
                               group_threads=256))
    r.run()
    pa = oracle_run(128, 40, 2, 0.1, 0.05, 77)
    pa.run()
    np.testing.assert_array_equal(r.population(), pa.pop)
    r.close()


def test_bad_arguments():
    for nbytes, tries in [(8, 10), (4100, 10), (24, 10), (64, 0)]:
        assert eng.selftest_bulk_wait(nbytes, True, tries) == "invalid argument"
