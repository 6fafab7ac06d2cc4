"""pa_gather, the replica copy of the resampling step as a standalone
kernel: new slot o holds old slot parent[o], word for word (checked against
numpy fancy indexing, the definition of the copy)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402


def resample_like_parents(n_old, seed):
    """Sorted parents with copy numbers 0..3 around a mean of 1, as the
    nearest-integer resampling produces them."""
    rng = np.random.default_rng(seed)
    r = rng.choice(4, size=n_old, p=[0.3, 0.45, 0.2, 0.05])
    return np.repeat(np.arange(n_old), r).astype(np.int32)


@pytest.mark.parametrize("n_old,words", [(1, 4), (37, 8), (1000, 128), (3001, 512), (777, 2048)])
def test_gather_matches_indexing(n_old, words):
    rng = np.random.default_rng(n_old + words)
    src = rng.integers(-2 ** 31, 2 ** 31, size=n_old * words, dtype=np.int64).astype(np.int32)
    parent = resample_like_parents(n_old, words)
    if parent.size == 0:
        parent = np.zeros(1, dtype=np.int32)
    dst, ms = eng.gather(torch.from_numpy(src).cuda(), torch.from_numpy(parent).cuda(), words)
    want = src.reshape(n_old, words)[parent].ravel()
    np.testing.assert_array_equal(dst.cpu().numpy(), want)
    assert ms >= 0.0


def test_gather_rejects_parent_outside_source():
    words, n_old = 8, 50
    src = np.arange(n_old * words, dtype=np.int32)
    parent = np.array([0, 3, n_old, 7], dtype=np.int32)  # one index past the source
    dst = torch.full((parent.size * words,), -5, dtype=torch.int32, device="cuda")
    with pytest.raises(eng.PAError) as ei:
        eng.gather(torch.from_numpy(src).cuda(), torch.from_numpy(parent).cuda(), words, dst=dst)
    assert ei.value.kind == "invalid argument"
    got = dst.cpu().numpy().reshape(parent.size, words)
    for o, p in enumerate(parent):
        if p < n_old:
            np.testing.assert_array_equal(got[o], src.reshape(n_old, words)[p])
        else:
            assert (got[o] == -5).all()  # skipped: nothing written
