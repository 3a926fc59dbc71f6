"""The library built with the device bounds checks (PDN_CHECK, loaded with
PDN_CHECKED=1): every element's node ids and every contact-surface node are
checked on the device before use, a failure recorded in the control block
halts the run.  On valid meshes the checked build runs clean and gives the
same states as the regular build (a plain FP64 impact, and an FP32 impact
with damage and interfaces on box hexes and flat interfaces), each build in a
child process of its own."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import pdn_inputs as pi

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
import paper_2301_05552_gb300 as pkg
import pdn_inputs as pi
L = pkg.lib()
out = {{"lib": L._name}}
for name, w, n in (("fp64", pi.plain_fp64_plate(nx=16, ny=16, steps=400), 400),
                   ("fp32", pi.damage_fp32_plate(nx=24, ny=36, plies=8, Lx=12.5, Ly=18.75, H=2.2,
                                                 mass=5.5e-3 / 64, speed=20000.0, steps=700), 700)):
    g = pkg.Solver(w)
    g.step(n)
    d, v, _ = g.state()
    out[name] = {{"d": d.ravel().tolist(), "f": g.force_history().tolist(), "status": pkg.pdn_get_info(g.ctx)["status"]}}
    g.close()
print(json.dumps(out))
"""


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env.setdefault("PDN_HEX_VARIANT", "0")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], capture_output=True, text=True, env=env,
                       timeout=1200)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_runs_clean_and_matches():
    chk = _run({"PDN_CHECKED": "1"})
    reg = _run({"PDN_CHECKED": "0"})
    assert chk["lib"].endswith("libpdn_check.so") and reg["lib"].endswith("libpdn.so")
    for name in ("fp64", "fp32"):
        a, b = chk[name], reg[name]
        assert a["status"] == 0 and b["status"] == 0
        da, db = np.array(a["d"]), np.array(b["d"])
        fa, fb = np.array(a["f"]), np.array(b["f"])
        assert fb.max() > 0.0, "the run must reach contact"
        tol = 1e-12 if name == "fp64" else 1e-6
        assert np.abs(da - db).max() <= tol * np.abs(db).max()
        assert np.abs(fa - fb).max() <= tol * np.abs(fb).max()
