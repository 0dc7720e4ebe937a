"""The C ABI library builds, loads and exports every entry point that
include/air.h declares; no GPU needed."""
import os
import re

import paper_2010_11130_gb300 as air
from paper_2010_11130_gb300.air import EXPORTED

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "air.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(air_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_binding_names():
    assert sorted(EXPORTED) == _declared()


def test_library_exports_every_declared_symbol():
    air.build()
    L = air.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_status_strings_and_defaults():
    assert air.status_string(0) == "ok"
    assert "iteration cap" in air.status_string(-6)
    o = air.default_options()
    assert abs(o.theta - 0.25) < 1e-15 and o.relax == b"FCF" and o.restart == 30
