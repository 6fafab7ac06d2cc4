"""Batched runs (pa_batch_*): every run of a batch gives the same results as
the same configuration run alone, bit for bit, whatever the threads per
replica chosen for it (warp groups or one replica per CTA), after a reset
with new seeds, and when another run of the batch fails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from tests._parity import assert_row_close, oracle_run  # noqa: E402

B32 = eng.SPIN_BITS32

MIX = [
    # L, R, theta, beta_f, dbeta, seed  (uneven sizes and step counts)
    (64, 2600, 3, 0.3, 0.05, 101),
    (16, 1500, 5, 0.5, 0.05, 102),
    (8, 700, 2, 0.2, 0.05, 103),
    (128, 300, 2, 0.2, 0.1, 104),
    (32, 1100, 4, 0.4, 0.05, 105),
    (256, 40, 1, 0.3, 0.15, 106),
    (16, 3000, 2, 0.25, 0.05, 107),
]


def cfg(L, R, theta, beta_f, dbeta, seed, **kw):
    return eng.PAConfig(L=L, R=R, theta=theta, beta_f=beta_f, dbeta=dbeta, seed=seed, spin_format=B32,
                        record_histograms=True, **kw)


def alone(c):
    r = eng.PARun(eng.PAConfig(**{**c.__dict__, "group_threads": 0}))
    r.run()
    out = (r.rows(), r.population(), r.histogram(0, 2))
    r.close()
    return out


def check_same(batch, refs):
    for i, (rows_ref, pop_ref, hsum_ref) in enumerate(refs):
        run = batch.runs[i]
        np.testing.assert_array_equal(run.rows(), rows_ref, err_msg=f"run {i} rows")
        np.testing.assert_array_equal(run.population(), pop_ref, err_msg=f"run {i} population")
        np.testing.assert_array_equal(run.histogram(0, 2), hsum_ref, err_msg=f"run {i} Hsum")


def test_batch_equals_alone_and_oracle():
    cfgs = [cfg(*m) for m in MIX]
    refs = [alone(c) for c in cfgs]
    b = eng.PABatch(cfgs)
    b.run()
    check_same(b, refs)
    # and the small ones against the oracle directly
    for i in (1, 2):
        L, R, theta, beta_f, dbeta, seed = MIX[i]
        pa = oracle_run(L, R, theta, beta_f, dbeta, seed)
        pa.run()
        rows = b.runs[i].rows()
        for j, ref in enumerate(pa.rows):
            assert_row_close(rows[j], ref, f"batch run {i} row {j}")
        np.testing.assert_array_equal(b.runs[i].population(), pa.pop)
    b.close()


def test_batch_with_a_large_population():
    """A run whose capacity is above the one-CTA resampling limit (16384)
    takes the batch through the multi-kernel bookkeeping (tables, counts,
    scan, parents, statistics: one launch each for all runs); the small-run
    batches above take the one-CTA-per-run form. Both equal the runs alone."""
    mix = [(16, 16000, 1, 0.15, 0.05, 141), (32, 900, 2, 0.2, 0.05, 142), (128, 120, 1, 0.1, 0.05, 143),
           (8, 500, 3, 0.3, 0.05, 144)]
    cfgs = [cfg(*m) for m in mix]
    refs = [alone(c) for c in cfgs]
    b = eng.PABatch(cfgs)
    b.run()
    check_same(b, refs)
    b.close()


def test_batch_group_shapes_do_not_change_results():
    base = [cfg(*m) for m in MIX[:5]]
    refs = [alone(c) for c in base]
    shapes = {64: 16, 16: 2, 8: 1, 128: 32, 32: 8}
    b = eng.PABatch([cfg(*m, group_threads=shapes[m[0]]) for m in MIX[:5]])
    for i, m in enumerate(MIX[:5]):
        assert b.shape(i)["group_threads"] == shapes[m[0]]
    b.run()
    check_same(b, refs)
    b.close()


def test_batch_cta_groups_mixed_with_warp_groups():
    """Runs with one replica per 256-thread CTA (L >= 128, including L = 512,
    which has no warp-group shape) are taken first by whole CTAs, the rest
    by warps, in the same launch; every run is bit-identical to itself run
    alone."""
    mix = [(128, 300, 2, 0.2, 0.1, 111), (64, 900, 2, 0.2, 0.1, 112), (512, 24, 1, 0.2, 0.1, 113),
           (16, 700, 3, 0.3, 0.1, 114), (256, 60, 1, 0.3, 0.15, 115), (32, 400, 2, 0.2, 0.1, 116)]
    shapes = {128: 256, 64: 32, 512: 256, 16: 4, 256: 256, 32: 16}
    refs = [alone(cfg(*m)) for m in mix]
    b = eng.PABatch([cfg(*m, group_threads=shapes[m[0]]) for m in mix])
    for i, m in enumerate(mix):
        assert b.shape(i)["group_threads"] == shapes[m[0]]
    b.run()
    check_same(b, refs)
    b.close()


def test_batch_of_cta_group_runs_only():
    mix = [(128, 200, 2, 0.2, 0.1, 121), (256, 30, 1, 0.2, 0.1, 122), (128, 77, 3, 0.3, 0.1, 123)]
    refs = [alone(cfg(*m)) for m in mix]
    b = eng.PABatch([cfg(*m, group_threads=256) for m in mix])
    b.run()
    check_same(b, refs)
    b.close()


def test_batch_rejects_unsupported_group_shape():
    with pytest.raises(eng.PAError):
        eng.PABatch([cfg(64, 100, 1, 0.1, 0.1, 1, group_threads=256)])
    with pytest.raises(eng.PAError):
        eng.PABatch([cfg(512, 10, 1, 0.1, 0.1, 1, group_threads=32)])


def test_batch_reset_with_new_seeds():
    cfgs = [cfg(*m) for m in MIX[:4]]
    b = eng.PABatch(cfgs)
    b.run()
    seeds = [900 + i for i in range(4)]
    b.reset(seeds)
    b.run()  # graph replay
    refs = [alone(eng.PAConfig(**{**c.__dict__, "seed": s})) for c, s in zip(cfgs, seeds)]
    check_same(b, refs)
    b.close()


def test_one_failing_run_leaves_the_others():
    good = [cfg(*m) for m in MIX[:3]]
    bad = cfg(8, 500, 1, 1.0, 0.2, 3, capacity=500)
    refs = [alone(c) for c in good]
    b = eng.PABatch(good + [bad])
    with pytest.raises(eng.PAError) as ei:
        b.run()
    assert ei.value.kind == "capacity"
    check_same(b, refs)
    b.close()


def test_failing_cta_group_run_leaves_the_others():
    """A run of one replica per CTA (swept by its own kernel inside the
    batch) that exceeds its capacity stops there; the warp-group and
    CTA-group runs beside it equal their runs alone."""
    good = [cfg(128, 200, 2, 0.3, 0.1, 131), cfg(32, 600, 2, 0.3, 0.1, 132), cfg(256, 40, 1, 0.3, 0.1, 133)]
    bad = cfg(128, 64, 1, 1.0, 0.25, 134, capacity=64, group_threads=256)
    refs = [alone(c) for c in good]
    b = eng.PABatch(good + [bad])
    assert b.shape(3)["group_threads"] == 256
    with pytest.raises(eng.PAError) as ei:
        b.run()
    assert ei.value.kind == "capacity"
    check_same(b, refs)
    b.close()


def test_config4_draw_matches_oracle_philox():
    from oracle.pa_oracle import philox_many
    got = eng.batch_config4_draw(64)
    ctr = np.zeros((64, 4), dtype=np.uint32)
    ctr[:, 1] = np.arange(64)
    ctr[:, 2] = 3
    w = philox_many(ctr, 99)
    for r in range(64):
        L = [16, 32, 64, 128][int(w[r, 0]) % 4]
        R = 2000 + int(w[r, 1]) % 48001
        th = [10, 50, 100][int(w[r, 2]) % 3]
        assert got[r] == (L, R, th)
