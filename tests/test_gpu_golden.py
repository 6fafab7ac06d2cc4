"""The engine against the stored oracle fixtures of tests/golden/ (written by
tests/golden/make_golden.py from oracle/ only): config 1 in both
single-spin formats, the simple cubic run and a 3-state Potts run, every
row within 1e-12 of the
stored one, R_i and family counts equal, the final population's FNV-1a 64
hash equal."""
import math

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1703_03676_gb300 as eng  # noqa: E402
from tests.golden.make_golden import ROW_FIELDS, read_rows  # noqa: E402

CASES = [("oracle_rows_config1.txt", eng.SPIN_BITS32), ("oracle_rows_config1.txt", eng.SPIN_INT8),
         ("oracle_rows_3d_L8.txt", eng.SPIN_BITS32), ("oracle_rows_potts_q3_L16.txt", eng.SPIN_INT8)]


@pytest.mark.parametrize("name,fmt", CASES, ids=["config1-bits", "config1-int8", "3d-L8", "potts-q3-L16"])
def test_engine_matches_stored_rows(name, fmt):
    p, h, rows = read_rows(name)
    run = eng.PARun(eng.PAConfig(L=p["L"], R=p["R"], theta=p["theta"], beta_f=p["beta_f"], dbeta=p["dbeta"],
                                 seed=p["seed"], spin_format=fmt, dim=p["dim"], potts_q=p.get("potts_q", 0)))
    run.run()
    got = run.rows()
    assert len(got) == len(rows)
    for i, ref in enumerate(rows):
        for k in ROW_FIELDS:
            a, b = float(got[k][i]), ref[k]
            if k in ("R", "families"):
                assert a == b, (name, i, k)
            else:
                assert a == b or math.isclose(a, b, rel_tol=1e-12, abs_tol=1e-300), (name, i, k, a, b)
    assert run.population_hash() == h
    run.close()
