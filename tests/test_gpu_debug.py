"""The debug build of the library (POND_DEBUG: index checks on the staged
kernel's global and shared-memory accesses that count a failure and skip
the access, never trapping), exercised where index arithmetic is most
fragile: 1 x 1 to 4 x 4 periodic grids, whose stencils and staged windows
wrap around the grid many times, plus a ragged 37 x 29 grid.  Every check
must pass (index_faults == 0) and the results must equal the release
library's to rounding.

The debug library runs in a child process (the binding loads one library
per process); it writes its results to a file the test compares."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1806_05089_gb300 import build, pond, workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [(1, 1), (2, 1), (1, 3), (3, 2), (4, 4), (37, 29)]
FORMS = [("fp64", pond.POND_FP64, pond.POND_D2Q16), ("mixed", pond.POND_FP32_MIXED, pond.POND_D2Q16),
         ("fp64_q9", pond.POND_FP64, pond.POND_D2Q9), ("mixed_q9", pond.POND_FP32_MIXED, pond.POND_D2Q9)]

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1806_05089_gb300 import pond
from tests.test_gpu_debug import run_all
pond.load(path=sys.argv[2])
json.dump(run_all(), open(sys.argv[3], "w"))
"""


def run_all():
    out = {}
    for name, prec, lat in FORMS:
        T_L = 1.0 / 3.0 if lat == pond.POND_D2Q9 else 1.0
        for nx, ny in CASES:
            f = workloads.supersonic(nx=nx, ny=ny)
            f.T, f.ux, f.uy = f.T * T_L, f.ux * T_L ** 0.5, f.uy * T_L ** 0.5
            for ty in ((4, 8) if prec == pond.POND_FP64 else (4, 8, 16)):
                with pond.Sim(nx, ny, prec, lattice=lat, T_ref=T_L, tile_rows=ty) as s:
                    s.set_state(f.rho, f.ux, f.uy, f.T)
                    st = s.step(3)
                    rho, ux, uy, T = s.moments()
                out["%s_%dx%d_ty%d" % (name, nx, ny, ty)] = {
                    "faults": int(st["index_faults"]), "nonphysical": int(st["nonphysical"]),
                    "rho": rho.tolist(), "T": T.tolist(), "ux": ux.tolist()}
    return out


def test_debug_build_index_checks_pass_on_tiny_and_ragged_grids(tmp_path):
    lib = build.build(debug=True)
    res = tmp_path / "debug.json"
    subprocess.run([sys.executable, "-c", CHILD, ROOT, lib, str(res)], check=True, cwd=ROOT,
                   timeout=600)
    dbg = json.load(open(res))
    rel = run_all()
    assert set(dbg) == set(rel)
    for key, d in dbg.items():
        assert d["faults"] == 0, key
        assert d["nonphysical"] == 0, key
        r = rel[key]
        tol = 1e-12 if key.startswith("fp64") else 1e-6
        for fld in ("rho", "T", "ux"):
            a, b = np.array(d[fld]), np.array(r[fld])
            assert np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max()), (key, fld)
