"""FP32 element arithmetic against the FP64 oracle on the full-size plates
that the benchmark times (element forces, damage and cohesive law in FP32;
integration, striker and gap test in FP64).

* 100x150x4.4 mm plate, 128x192x16 hex8, 5.5 kg at 3 m/s: both solvers from
  rest through first contact (about 400 steps) and 1,600 steps of contact,
  into the first matrix damage under the striker.
  Contact-force history within 0.5 % of its peak at every step, peak force
  within 0.5 %, displacements within 1e-4 of the largest.
* 400x600x32 hex8 refinement (7.68 M hex), 5.5 kg at 4 m/s: the GPU steps
  through its pre-roll into the contact phase; its committed state
  (displacement, velocity, acceleration, Gauss-point and interface history,
  contact set, striker) is installed in the oracle, and both advance 20
  steps.  Contact force within 0.5 % at every step, displacements within
  1e-4, thresholds within 1e-3, velocity increments within 1e-2 (the
  velocity field carries the high-frequency part of the FP32 rounding
  differences of the nodal forces; 1.7e-3 measured).

The measured errors are printed (pytest -s) beside the asserted bounds.
"""
import os

import numpy as np
import pytest

import oracle
import pdn_inputs as pi

pytestmark = pytest.mark.gpu

F32_PEAK_TOL = 5e-3
F32_DISP_TOL = 1e-4


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _threads():
    return len(os.sched_getaffinity(0))


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_fp32_damage_plate_from_rest_through_contact(pkg):
    w = pi.damage_fp32_plate()
    g = pkg.Solver(w)
    o = oracle.model_for(w, n_threads=_threads())
    n = 2000
    for _ in range(n // 100):
        g.step(100)
        assert o.step(100) == 0
    fg, fo = g.force_history(), o.force_history()
    assert len(fg) == len(fo) == n
    first = int(np.argmax(fo > 0.0))
    assert fo.max() > 0.0 and first < n - 1000, "the window must reach well into contact"
    f_err = float(np.abs(fg - fo).max() / fo.max())
    pk_err = abs(fg.max() - fo.max()) / fo.max()
    dg, _, _ = g.state()
    do, _, _ = o.state()
    d_err = _rel(dg, do)
    hist, rD = o.history()
    damaged = int((hist[:, :, :4] > 1.0).any(axis=(1, 2)).sum())
    print(f"\n100x150 plate, {n} steps from rest: first contact at step {first + 1}, peak {fo.max():.2f} N, "
          f"force history err {f_err:.2e} of peak, peak err {pk_err:.2e}, displacement err {d_err:.2e}, "
          f"damaged hexes {damaged}, damaged interfaces {int((rD > 0).any(axis=1).sum())}")
    assert damaged > 0, "the window must reach damage"
    assert pk_err <= F32_PEAK_TOL
    assert f_err <= F32_PEAK_TOL
    assert d_err <= F32_DISP_TOL
    g.close()
    o.close()


def test_fp32_large_plate_loaded_state_continued_by_oracle(pkg):
    w = pi.large_fp32_plate()
    assert w.preroll > 0
    g = pkg.Solver(w)
    g.step(w.preroll)
    info = g.info()
    assert info["n_active"] > 0, "the pre-roll must end in contact"
    d0, v0, imp = g.state()
    a0 = pkg.pdn_get_acceleration(g.ctx)
    act, _ = pkg.pdn_get_contact(g.ctx)
    hist, rD = pkg.pdn_get_history(g.ctx)
    damaged0 = int((hist[:4] > 1.0).any(axis=(0, 1)).sum())
    o = oracle.model_for(w, n_threads=_threads())
    o.set_history(hist.astype(np.float64).transpose(2, 1, 0), rD.astype(np.float64).T)
    o.install_state(d0, v0, a0, act, imp, info["step"])
    del hist, rD
    k = 20
    g.step(k)
    assert o.step(k) == 0
    fg = g.force_history()[-k:]
    fo = o.force_history()
    assert len(fo) == k and fo.min() > 0.0
    f_err = float(np.abs(fg - fo).max() / np.abs(fo).max())
    dg, vg, _ = g.state()
    do, vo, _ = o.state()
    d_err = _rel(dg, do)
    dv_err = _rel(vg - v0, vo - v0)
    hg, rg = pkg.pdn_get_history(g.ctx)
    ho, ro = o.history()
    r_err = _rel(hg[:4].astype(np.float64), ho[:, :, :4].transpose(2, 1, 0))
    ag, _ = pkg.pdn_get_contact(g.ctx)
    ao, _ = o.active()
    sym = int(np.count_nonzero(ag != ao))
    print(f"\n400x600x32 plate, step {info['step']} (contact nodes {info['n_active']}, damaged hexes {damaged0}) "
          f"+ {k} steps: force err {f_err:.2e} of max, displacement err {d_err:.2e}, velocity-increment err "
          f"{dv_err:.2e}, threshold err {r_err:.2e}, contact-set differences {sym} of {int(ao.sum())}")
    assert f_err <= F32_PEAK_TOL
    assert d_err <= F32_DISP_TOL
    assert dv_err <= 1e-2
    assert r_err <= 1e-3
    assert sym <= max(2, int(0.02 * ao.sum()))
    g.close()
    o.close()
