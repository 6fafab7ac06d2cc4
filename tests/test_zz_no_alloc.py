"""pa_resample_noalloc, the allocation-free form of pa_resample.

Callers such as a memory-budgeted server or a program whose device memory
belongs to another allocator cannot let the library call cudaMalloc once
they are running; this entry point keeps its scratch in a static device
array instead. It must give exactly what pa_resample gives. The file is
named to be collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from tests.test_gpu_resample import oracle_case  # noqa: E402


def _call(lev, F, U, seed, step, cap, noalloc):
    return eng.resample(torch.from_numpy(lev.astype(np.int32)).cuda(),
                        torch.from_numpy(F.astype(np.uint32).view(np.int32)).cuda(),
                        torch.from_numpy(U).cuda(), seed, step, cap, noalloc=noalloc)


def test_noalloc_matches_allocating_entry_point_twice():
    # two calls in a row: the second must not see the first one's scratch
    cases = [(70001, 0.005, 77, 9), (3000, 0.03, 5, 2)]
    for n_old, delta, seed, step in cases:
        lev, F, U, parent = oracle_case(n_old, 4096, seed, step, delta, n_old)
        cap = 2 * n_old + 16
        ref, n_ref = _call(lev, F, U, seed, step, cap, noalloc=False)
        got, n_got = _call(lev, F, U, seed, step, cap, noalloc=True)
        assert n_got == n_ref == parent.size
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_after_a_failed_call_and_at_the_size_limit():
    # a call that leaves a capacity status in the shared array, then good
    # calls: the status word is cleared and every other part of the scratch
    # is written before it is read, so they must match pa_resample
    lev, F, U, parent = oracle_case(3000, 4096, 5, 3, 0.05, 3000)
    with pytest.raises(eng.PAError) as ei:
        _call(lev, F, U, 5, 3, parent.size - 1, noalloc=True)
    assert ei.value.kind == "capacity"
    n_old = eng.RESAMPLE_NOALLOC_MAX_OLD  # the largest population the array holds
    for n, seed, step in [(2000, 11, 4), (n_old, 12, 7)]:
        lev, F, U, parent = oracle_case(n, 4096, seed, step, 0.004, n)
        cap = 2 * n + 16
        ref, n_ref = _call(lev, F, U, seed, step, cap, noalloc=False)
        got, n_got = _call(lev, F, U, seed, step, cap, noalloc=True)
        assert n_got == n_ref == parent.size
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
        np.testing.assert_array_equal(got.cpu().numpy(), parent)


def test_noalloc_rejects_oversize():
    n_old = eng.RESAMPLE_NOALLOC_MAX_OLD + 1
    lev = torch.zeros(n_old, dtype=torch.int32, device="cuda")
    F = torch.ones(8, dtype=torch.int32, device="cuda")
    U = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(eng.PAError) as ei:
        eng.resample(lev, F, U, 1, 1, n_old + 10, noalloc=True)
    assert ei.value.kind == "invalid argument"
    assert b"exceeds the static scratch limit" in eng.lib().pa_last_error_message()
