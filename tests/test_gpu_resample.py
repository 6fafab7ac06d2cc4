"""Kernel-level resampling entry point (pa_resample) against the oracle's
copy numbers (Eq. resampling-factors) on the same levels, tables and
RESAMPLE stream: the parent list must match exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from oracle.pa_oracle import copy_tables, level_weights, normaliser_S, resample_words  # noqa: E402


def oracle_case(n_old, N, seed, step, delta, R):
    rng = np.random.default_rng(seed)
    lev = np.clip(np.round(rng.normal(N * 0.3, N * 0.05, n_old)), 0, N).astype(np.int64)
    H = np.bincount(lev, minlength=N + 1)
    kmin, kmax = int(lev.min()), int(lev.max())
    t = level_weights(delta, kmax - kmin + 1)
    S = normaliser_S(H, kmin, kmax, t, N)
    _, Fd, Ud = copy_tables(R, t, S)
    F = np.zeros(N + 1, dtype=np.int64)
    U = np.zeros(N + 1, dtype=np.int64)
    F[kmin:kmax + 1] = Fd
    U[kmin:kmax + 1] = Ud
    x = resample_words(seed, step, n_old).astype(np.int64)
    r = F[lev] + (x < U[lev])
    parent = np.repeat(np.arange(n_old), r)
    return lev, F, U, parent


@pytest.mark.parametrize("n_old,delta", [(1, 0.0), (1000, 0.01), (5000, 0.02), (70001, 0.005)])
def test_resample_matches_oracle(n_old, delta):
    N, seed, step = 4096, 77, 9
    R = n_old
    lev, F, U, parent = oracle_case(n_old, N, seed, step, delta, R)
    got, n = eng.resample(torch.from_numpy(lev.astype(np.int32)).cuda(),
                          torch.from_numpy(F.astype(np.uint32).view(np.int32)).cuda(),
                          torch.from_numpy(U).cuda(), seed, step, 2 * n_old + 16)
    assert n == parent.size
    np.testing.assert_array_equal(got.cpu().numpy(), parent)


def test_resample_capacity_error():
    N, seed, step = 4096, 5, 3
    lev, F, U, parent = oracle_case(3000, N, seed, step, 0.05, 3000)
    with pytest.raises(eng.PAError) as ei:
        eng.resample(torch.from_numpy(lev.astype(np.int32)).cuda(),
                     torch.from_numpy(F.astype(np.uint32).view(np.int32)).cuda(),
                     torch.from_numpy(U).cuda(), seed, step, parent.size - 1)
    assert ei.value.kind == "capacity"


@pytest.mark.parametrize("noalloc", [False, True])
def test_resample_wrapping_copy_numbers_rejected(noalloc):
    """Caller tables whose copy numbers sum past 2^32: F = 2^31 for two slots
    and 1 for a third give R_i = 2^32 + 1, which a 32-bit total would wrap
    to 1 and accept. The call must report the capacity error and leave the
    parent buffer unwritten."""
    F = np.array([2 ** 31, 1], dtype=np.int64)
    lev = np.array([0, 0, 1], dtype=np.int64)
    total = int(sum(int(F[k]) for k in lev))  # exact, on the CPU
    assert total == 2 ** 32 + 1 and total % 2 ** 32 == 1
    cap = 8
    parent = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(eng.PAError) as ei:
        eng.resample(torch.from_numpy(lev.astype(np.int32)).cuda(),
                     torch.from_numpy(F.astype(np.uint32).view(np.int32)).cuda(),
                     torch.zeros(2, dtype=torch.int64, device="cuda"), 3, 1, cap, parent=parent, noalloc=noalloc)
    assert ei.value.kind == "capacity"
    assert bool((parent == -7).all())


def test_resample_capacity_over_tiles_leaves_parent_unwritten():
    """A ragged population of 2500 slots (three tiles) whose tiles each fit
    the capacity but whose total does not: capacity error, nothing written."""
    n_old = 2500
    lev = np.zeros(n_old, dtype=np.int64)
    F = np.array([3], dtype=np.int64)
    cap = 4000  # each tile holds at most 1024 * 3 = 3072 copies; the total is 7500
    parent = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(eng.PAError) as ei:
        eng.resample(torch.from_numpy(lev.astype(np.int32)).cuda(),
                     torch.from_numpy(F.astype(np.uint32).view(np.int32)).cuda(),
                     torch.zeros(1, dtype=torch.int64, device="cuda"), 9, 2, cap, parent=parent)
    assert ei.value.kind == "capacity"
    assert bool((parent == -7).all())
