"""Write the oracle-derived golden fixtures of tests/golden/.

Every value here comes from oracle/ (the plain CPU statement of the method
and the exact Ising references); nothing is computed by the CUDA engine.
Re-run after a change to the oracle's arithmetic, in the same commit, whose
message names the passage of the paper (or the reading of it) that
justifies the change:

    python tests/golden/make_golden.py

Fixtures:
  exact_dos.txt               exact g(E): 4 x 4 and 2 x 2 x 2 tori by
                              enumeration, 6 x 6 and the 3-state Potts
                              4 x 4 torus by transfer matrix
  oracle_rows_config1.txt     config 1 (L = 16, R = 1000, theta = 10,
                              dbeta = 0.01 to beta = 1, seed 1): every row
                              and the final population's FNV-1a 64 hash
  oracle_rows_3d_L8.txt       simple cubic L = 8, R = 500, theta = 3,
                              dbeta = 0.1 to beta = 0.6, seed 51
  oracle_rows_potts_q3_L16.txt  3-state Potts, L = 16, R = 500, theta = 5,
                              dbeta = 0.1 to beta = 1.2, seed 61
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact_ising import BruteForce, potts_transfer_dos, transfer_matrix_dos  # noqa: E402
from oracle.pa_oracle import PopulationAnnealing  # noqa: E402

ROW_FIELDS = ["beta", "e", "C", "abs_m", "m2", "m4", "betaF_per_N", "S_per_N", "lnQ", "R", "families"]

RUNS = {
    "oracle_rows_config1.txt": dict(L=16, R=1000, theta=10, beta_f=1.0, dbeta=0.01, seed=1, dim=2),
    "oracle_rows_3d_L8.txt": dict(L=8, R=500, theta=3, beta_f=0.6, dbeta=0.1, seed=51, dim=3),
    "oracle_rows_potts_q3_L16.txt": dict(L=16, R=500, theta=5, beta_f=1.2, dbeta=0.1, seed=61, dim=2, potts_q=3),
}


def fnv1a64(spins) -> int:
    """64-bit FNV-1a over int8 spins (+1/-1, or Potts states), one byte each,
    in natural layout."""
    h = 0xCBF29CE484222325
    for v in spins.astype("int8").ravel().view("uint8").tolist():
        h ^= v
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def run_rows(p):
    pa = PopulationAnnealing(p["L"], p["R"], p["theta"], beta_f=p["beta_f"], dbeta=p["dbeta"], seed=p["seed"],
                             dim=p["dim"], potts_q=p.get("potts_q", 0))
    pa.run()
    return pa.rows, fnv1a64(pa.pop)


def write_rows(name, p):
    rows, h = run_rows(p)
    with open(os.path.join(HERE, name), "w") as f:
        f.write("# written by tests/golden/make_golden.py from oracle.pa_oracle.PopulationAnnealing\n")
        f.write("# " + " ".join(f"{k}={v}" for k, v in p.items()) + "\n")
        f.write(f"# population_fnv1a64 {h}\n")
        f.write("# " + " ".join(ROW_FIELDS) + "\n")
        for r in rows:
            f.write(" ".join(repr(float(getattr(r, k))) if k not in ("R", "families") else str(getattr(r, k))
                             for k in ROW_FIELDS) + "\n")


def write_dos():
    tables = [("square L=4 (enumeration)", BruteForce(4).energy_dos()),
              ("square L=6 (transfer matrix)", transfer_matrix_dos(6)),
              ("cubic L=2 (enumeration)", BruteForce(2, dim=3).energy_dos()),
              ("potts q=3 L=4 (transfer matrix)", potts_transfer_dos(4, 3))]
    with open(os.path.join(HERE, "exact_dos.txt"), "w") as f:
        f.write("# written by tests/golden/make_golden.py from oracle.exact_ising\n")
        f.write("# lattice, then lines: E g(E)\n")
        for name, g in tables:
            f.write(f"lattice {name}\n")
            for e in sorted(g):
                f.write(f"{e} {g[e]}\n")


def read_rows(name):
    """(parameters, population hash, rows as dicts) of a rows fixture."""
    params, h, rows = {}, None, []
    with open(os.path.join(HERE, name)) as f:
        lines = f.read().splitlines()
    for k, v in (kv.split("=") for kv in lines[1][2:].split()):
        params[k] = float(v) if "." in v else int(v)
    h = int(lines[2].split()[2])
    for ln in lines[4:]:
        vals = ln.split()
        rows.append({k: (int(v) if k in ("R", "families") else float(v)) for k, v in zip(ROW_FIELDS, vals)})
    return params, h, rows


def read_dos():
    out, cur = {}, None
    with open(os.path.join(HERE, "exact_dos.txt")) as f:
        for ln in f:
            if ln.startswith("#"):
                continue
            if ln.startswith("lattice "):
                cur = ln[len("lattice "):].strip()
                out[cur] = {}
            else:
                e, g = ln.split()
                out[cur][int(e)] = int(g)
    return out


def read_paper_values():
    out = {}
    with open(os.path.join(HERE, "paper_values.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            key, value = ln.split()[:2]
            out[key] = value
    return out


if __name__ == "__main__":
    write_dos()
    for name, p in RUNS.items():
        write_rows(name, p)
    print("wrote", ", ".join(["exact_dos.txt"] + list(RUNS)))
