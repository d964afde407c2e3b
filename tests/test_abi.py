"""The C ABI library loads without a GPU and exports every entry point include/lmood.h declares."""
import os
import re

import paper_2104_02139_gb300 as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lmood.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(lmood_[a-z_]+)\s*\(", src))


def test_header_and_exports_agree():
    L.build()
    lib = L.lib()
    declared = _declared()
    assert declared == set(L.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_params_default_without_gpu():
    p = L.params_default(3)
    assert p.cfl == 0.25 and p.Cv == 0.2 and p.Ci == 0.1 and p.delta0 == 1e-4 and p.delta1 == 1e-3
    assert p.order == 2 and p.mood == 1 and p.max_mood_iters == 100000
    try:
        L.params_default(4)
    except L.LmoodError as e:
        assert e.status == L.ERR_ARG
    else:
        raise AssertionError("dim 4 accepted")
