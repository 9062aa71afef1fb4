"""Bounds-checked build of the library (LBM_BOUNDS_CHECK): every population,
frame and porosity access of the step kernels' pull, wall rule and stores is
checked against its plane before it is made, and one outside is skipped and
counted (lbm_bounds_check).  A stand-in for a memory checker on small and
odd-sized lattices, where the pull's x and y shifts meet the plane edges:
every precision, launch mode and wall variant, the porosity field, the
observing steps, the adjoint's recomputation and the batched kernel's tile
kinds must run with no access outside its plane.

The test builds the checked library (a second copy of the sources compiled
with LBM_BOUNDS_CHECK) and runs it in a child process, so that the normal
library of this process is left alone."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes as C
import json
import sys

sys.path.insert(0, sys.argv[1])
from paper_1308_2071_gb300 import _lib

lib = _lib.load(sys.argv[2])
import torch

from paper_1308_2071_gb300 import Batch, Cavity

torch.cuda.set_device(0)


def count():
    en, n = C.c_int(), C.c_long()
    _lib.check(lib.lbm_bounds_check(C.byref(en), C.byref(n)))
    return en.value, n.value


enabled, _ = count()
runs = []
for (nx, ny) in [(8, 8), (16, 16), (17, 13), (7, 9), (5, 5), (6, 11)]:
    for prec in ("f64", "f32", "f16", "f32t"):
        for npt in (1, 2, 3):
            for kw in ({}, dict(adiabatic_order=2), dict(thermal_bc=1, RaI=1e4), "field"):
                extra = {} if kw == "field" else kw
                phi = torch.full((ny, nx), 0.55, dtype=torch.float64, device="cuda") if kw == "field" else None
                c = Cavity(nx, ny, Ra=1e5, Da=1e-2, phi=0.6, precision=prec, nodes_per_thread=npt, block_x=32,
                           block_y=2, phi_field=phi, **extra)
                c.step(7)
                c.step_nusselt(3)
                c.observables(fields=True)
                c.read_state()
                c.extrema()
                if kw == "field" and prec in ("f64", "f32", "f32t"):
                    c.adjoint(12, 5)
                c.close()
                runs.append([nx, ny, prec, npt, str(kw), count()[1]])
for tw, th in ((32, 1), (32, 2), (32, 0), (256, 0), (32, -1), (256, -1)):
    cavs = [dict(nx=n, ny=m, Ra=1e4, Da=1e-2, phi=0.6) for (n, m) in ((5, 7), (9, 9), (17, 13), (33, 6))]
    b = Batch(cavs, precision="f32")
    b.set_tiles(tw, th, 0, 1)
    b.step(9)
    b.nusselt()
    b.close()
    runs.append(["batch", tw, th, count()[1]])
print(json.dumps(dict(enabled=enabled, runs=runs)))
"""


def test_no_access_leaves_its_plane_in_the_checked_build(tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_2071_gb300.build import build

    checked = build(checked=True)
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    r = subprocess.run([sys.executable, str(script), ROOT, checked], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["enabled"] == 1
    assert len(out["runs"]) == 6 * 4 * 3 * 4 + 6
    bad = [run for run in out["runs"] if run[-1] != 0]
    assert not bad, bad
