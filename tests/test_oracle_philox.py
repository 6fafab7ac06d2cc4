"""Pins for the oracle's Philox4x32-10 (Sec. 3 "Spin updates"; Salmon et al.
SC'11, the paper's generator).

The oracle's C implementation is compared with an independent third-party
implementation of the same published generator: Triton's ``tl.random.philox``
run in Triton's CPU interpreter. Statistical checks then confirm the words
are uniform and that the tagged streams used by the method are distinct.
"""
import os

import numpy as np
import pytest

from oracle.pa_oracle import philox4x32_10, philox_many, resample_words


def _triton_philox(seed, ctr):
    os.environ["TRITON_INTERPRET"] = "1"
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    import triton.language as tl

    @triton.jit
    def k(out_ptr, seed, c0_ptr, c1_ptr, c2_ptr, c3_ptr, n, BLOCK: tl.constexpr):
        i = tl.arange(0, BLOCK)
        m = i < n
        c0 = tl.load(c0_ptr + i, mask=m).to(tl.uint32)
        c1 = tl.load(c1_ptr + i, mask=m).to(tl.uint32)
        c2 = tl.load(c2_ptr + i, mask=m).to(tl.uint32)
        c3 = tl.load(c3_ptr + i, mask=m).to(tl.uint32)
        a, b, c, d = tl.random.philox(seed, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a.to(tl.int64) & 0xFFFFFFFF, mask=m)
        tl.store(out_ptr + 4 * i + 1, b.to(tl.int64) & 0xFFFFFFFF, mask=m)
        tl.store(out_ptr + 4 * i + 2, c.to(tl.int64) & 0xFFFFFFFF, mask=m)
        tl.store(out_ptr + 4 * i + 3, d.to(tl.int64) & 0xFFFFFFFF, mask=m)

    ctr = np.asarray(ctr, dtype=np.uint32).reshape(-1, 4)
    n = ctr.shape[0]
    block = 1
    while block < n:
        block *= 2
    cols = [torch.from_numpy(ctr[:, j].astype(np.int64)).to(torch.int32) for j in range(4)]
    out = torch.zeros(4 * n, dtype=torch.int64)
    k[(1,)](out, seed, cols[0], cols[1], cols[2], cols[3], n, BLOCK=block)
    return out.numpy().astype(np.uint64).reshape(n, 4)


def test_philox_matches_triton_interpreter():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2 ** 32, size=(61, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [5, 0, 0, 1]
    for seed in [0, 1, 2, 0xDEADBEEFCAFEF00D, 2 ** 64 - 1]:
        ours = philox_many(ctr, seed).astype(np.uint64)
        ref = _triton_philox(seed, ctr)
        np.testing.assert_array_equal(ours, ref)


def test_single_call_matches_batch():
    ctr = (3, 1, 4, 1)
    seed = 0x0000000500000009
    a = philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    b = philox_many(np.array([ctr], dtype=np.uint32), seed)[0]
    assert tuple(int(v) for v in b) == a


def test_philox_words_uniform():
    # 2^16 counters -> 2^18 words; chi^2 over 256 byte bins of every byte
    n = 1 << 16
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 1] = np.arange(n)
    ctr[:, 2] = 1
    w = philox_many(ctr, 12345).ravel()
    for shift in (0, 8, 16, 24):
        h = np.bincount(((w >> shift) & 0xFF).astype(np.int64), minlength=256)
        exp = w.size / 256
        chi2 = float(((h - exp) ** 2 / exp).sum())
        assert chi2 < 400, chi2  # 255 dof: mean 255, sd ~22.6
    # top bit unbiased: the INIT stream uses w < 2^31
    frac = float((w < 2 ** 31).mean())
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(w.size)


def test_streams_distinct():
    # resampling words of consecutive steps and the sweep stream tag differ
    a = resample_words(1, 1, 64)
    b = resample_words(1, 2, 64)
    c = resample_words(2, 1, 64)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    # lane layout: word j = lane j&3 of counter (i, j>>2, 2, 0)
    blk = philox_many(np.array([[1, 3, 2, 0]], dtype=np.uint32), 1)[0]
    np.testing.assert_array_equal(a[12:16], blk)
