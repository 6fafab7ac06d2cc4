"""The oracle's block-parallel form (workers > 1: contiguous blocks of
replicas on threads, each block run by the unchanged single-threaded C
routine) must give exactly what the serial form gives: every record, row,
histogram, copy number and the final population. It is what makes
full-size multi-step parity runs affordable."""
import numpy as np
import pytest

from oracle.pa_oracle import PopulationAnnealing, random_couplings

CASES = [
    dict(L=16, R=301, theta=3, beta_f=0.4, dbeta=0.05, seed=3),                    # fixed, ragged blocks
    dict(L=8, R=257, theta=2, beta_f=0.6, dbeta=0.0, seed=4, overlap=0.85),        # adaptive
    dict(L=8, R=200, theta=2, beta_f=0.3, dbeta=0.1, seed=5, msc=True),            # multi-spin-coded words
    dict(L=4, R=150, theta=3, beta_f=0.5, dbeta=0.1, seed=6, dim=3),               # simple cubic
    dict(L=8, R=120, theta=2, beta_f=0.6, dbeta=0.2, seed=7, potts_q=3),           # Potts
    dict(L=8, R=100, theta=2, beta_f=0.5, dbeta=0.1, seed=8, couplings=random_couplings(8, 1)),  # +-J
]


@pytest.mark.parametrize("kw", CASES, ids=["fixed", "adaptive", "msc", "cubic", "potts", "pmJ"])
def test_blocks_equal_serial(kw):
    a = PopulationAnnealing(**kw)
    a.run()
    b = PopulationAnnealing(**kw, workers=5)
    b.run()
    assert len(a.records) == len(b.records)
    for ra, rb in zip(a.records, b.records):
        assert (ra.R, ra.R_prev, ra.kmin_prev, ra.S, ra.delta, ra.beta, ra.families, ra.sums) == \
               (rb.R, rb.R_prev, rb.kmin_prev, rb.S, rb.delta, rb.beta, rb.families, rb.sums)
        np.testing.assert_array_equal(ra.H_E, rb.H_E)
        np.testing.assert_array_equal(ra.H_M, rb.H_M)
        if ra.counts is not None:
            np.testing.assert_array_equal(ra.counts, rb.counts)
    assert [r.as_tuple() for r in a.rows] == [r.as_tuple() for r in b.rows]
    np.testing.assert_array_equal(a.pop, b.pop)
    np.testing.assert_array_equal(a.fam, b.fam)
    np.testing.assert_array_equal(a.Hsum, b.Hsum)
    assert a.Msums == b.Msums
