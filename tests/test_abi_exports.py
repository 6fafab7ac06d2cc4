"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/pa.h declares (no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(pa_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    import paper_1703_03676_gb300 as eng
    L = eng.lib()
    names = declared_functions()
    assert len(names) >= 19, names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    bound = {s[0] for s in eng.SIGNATURES}
    assert set(names) <= bound | {"pa_footprint_bytes"}, set(names) - bound


def test_host_only_calls():
    import paper_1703_03676_gb300 as eng
    L = eng.lib()
    assert L.pa_strerror(-3) == b"population exceeded its capacity"
    cfg = eng.PAConfig(L=64, R=20000, theta=100, dbeta=0.005)
    fp = eng.footprint_bytes(cfg)
    # two ping-pong populations of 512 B per replica dominate
    assert 2 * 22024 * 512 < fp < 2 * 22024 * 512 + 8 * 22024 * 4 + 4_000_000
    bad = eng.PAConfig(L=7)
    assert eng.footprint_bytes(bad) == 0
