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
