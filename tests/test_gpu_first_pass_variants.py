"""Every first-pass kernel variant gives the same splitting.

The default cursor kernel falls back to the exact-bitmap kernel (variant 2)
and to the int32-measure kernels (variants 0 and 1) on levels outside its
limits; each variant is selected here for a whole setup in a child process
(the selection is read once per process) and must reproduce the default C/F
splitting of every level bit for bit.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import hashlib, json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_2010_11130_gb300 as air
from sthdg import assemble
from sthdg.problems import manufactured_2d
s = assemble(manufactured_2d(6, 2, 1e-6))
H = air.setup(air.CSR.from_host(s.row_ptr, s.col, s.val), theta=0.25, max_coarse=100)
print(json.dumps([hashlib.sha256(H.export(l, "cf").tobytes()).hexdigest() for l in range(H.levels() - 1)]))
"""


def _run(variant):
    env = dict(os.environ)
    if variant is None:
        env.pop("AIR_RS_VARIANT", None)
    else:
        env["AIR_RS_VARIANT"] = str(variant)
    code = _CHILD.replace("ROOT", repr(ROOT))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_variant_gives_the_default_splitting(variant):
    assert _run(variant) == _run(None)
