"""The column sweep (pdn_info.sweep, planned on request: PDN_SWEEP=1): one kernel evaluates the hexes and
interfaces of a tile of element columns layer by layer and updates the nodes
inside the tile from shared memory, in the gather's order; tile-boundary and
chunk-boundary nodes go through the element-force slots and a gather over
their list.  Against the separate element and gather kernels (PDN_SWEEP=0,
PDN_HEX_VARIANT=0 on both sides so that the same hex variant runs): the same
states to FP32 rounding (the two compile the element arithmetic in different
kernels; bitwise equal where they contract the same way), on plates whose
columns do not fill the tiles and with and without interfaces, through
contact, release and damage."""
import os

import numpy as np
import pytest

import oracle
import pdn_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _solver(pkg, w, sweep, monkeypatch):
    """A solver with the sweep (PDN_SWEEP=1, read at creation and by the first
    step) or without it (PDN_SWEEP=0), element variant 0 on both sides."""
    monkeypatch.setenv("PDN_HEX_VARIANT", "0")
    monkeypatch.setenv("PDN_SWEEP", "1" if sweep else "0")
    return pkg.Solver(w)


def _plates():
    out = []
    # interfaces, columns filling 8 x 4 tiles exactly, seeded damaging state
    w = pi.damage_fp32_plate(nx=32, ny=48, plies=8, Lx=12.5, Ly=18.75, H=2.2, steps=120)
    out.append(("interfaces_32x48x8", w, True))
    # ragged tiles (20 x 13 columns), two elements per ply, impact from rest
    w = pi.damage_fp32_plate(nx=20, ny=13, plies=4, elems_per_ply=2, Lx=10.0, Ly=6.5, H=1.1,
                             mass=5.5e-3 / 512, speed=20000.0, steps=900)
    out.append(("ragged_20x13x8", w, False))
    # no interfaces
    plate = pi.make_plate(12.0, 12.0, 2.0, 24, 24, [0.0, 90.0, 90.0, 0.0], 1, cohesive=False)
    mat = pi.material_im7_like_config(t_ply=0.5)
    w = pi.Workload("plain_fp32_24x24x4", plate, mat, False, True, True, 4.0, 1e-5, 10000.0, 0.01, 0.5, 900)
    out.append(("no_interfaces_24x24x4", w, False))
    return out


@pytest.mark.parametrize("name,w,seeded", _plates(), ids=[p[0] for p in _plates()])
def test_sweep_equals_separate_kernels(pkg, monkeypatch, name, w, seeded):
    a = _solver(pkg, w, True, monkeypatch)
    b = _solver(pkg, w, False, monkeypatch)
    assert pkg.pdn_get_info(a.ctx)["sweep"] > 0, "the sweep must be planned for this plate"
    assert pkg.pdn_get_info(b.ctx)["sweep"] == 0
    if seeded:
        Lx, Ly, H = w.plate.dims
        st = pi.seeded_state(w.plate, 7, amp=0.02, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.12, 1.5))
        pkg.pdn_set_state(a.ctx, *st)
        pkg.pdn_set_state(b.ctx, *st)
    monkeypatch.setenv("PDN_SWEEP", "1")
    a.step(w.steps)
    monkeypatch.setenv("PDN_SWEEP", "0")
    b.step(w.steps)
    assert pkg.pdn_get_info(a.ctx)["sweep"] > 0 and pkg.pdn_get_info(b.ctx)["sweep"] == 0
    da, va, _ = a.state()
    db, vb, _ = b.state()
    fa, fb = a.force_history(), b.force_history()
    ha, ra = pkg.pdn_get_history(a.ctx)
    hb, rb = pkg.pdn_get_history(b.ctx)
    bitwise = np.array_equal(da, db) and np.array_equal(fa, fb)
    print(f"\n{name}: sweep {pkg.pdn_get_info(a.ctx)['sweep']}, bitwise {bitwise}, "
          f"d {np.abs(da - db).max() / np.abs(db).max():.2e}, f peak {fb.max():.3f}, "
          f"repeats {pkg.pdn_get_info(a.ctx)['n_repeats']}/{pkg.pdn_get_info(b.ctx)['n_repeats']}")
    assert np.abs(da - db).max() <= 1e-6 * np.abs(db).max()
    assert np.abs(va - vb).max() <= 1e-4 * np.abs(vb).max()
    assert len(fa) == len(fb)
    if fb.max() > 0:
        assert np.abs(fa - fb).max() <= 1e-5 * fb.max()
    assert np.abs(ha.astype(np.float64) - hb).max() <= 1e-5 * max(np.abs(hb).max(), 1.0)
    if seeded:
        assert (hb[:4] > 1.0).any(), "the run must damage"
    else:
        assert fb.max() > 0.0, "the run must reach contact"
    a.close()
    b.close()


def test_sweep_against_oracle_through_release(pkg, monkeypatch):
    """The ragged plate with a light fast striker: contact, heavy damage and
    rebound with released nodes (Algorithm 2), the sweep against the FP64
    oracle: peak force within 0.5 %, the same number of repetitions, and
    displacements within 5e-3 of the largest (1.5e-3 measured after 3,000
    steps: softening damage amplifies the FP32 rounding of the element
    forces; the sweep is bitwise equal to the separate kernels, tested
    above)."""
    w = pi.damage_fp32_plate(nx=20, ny=13, plies=4, elems_per_ply=2, Lx=10.0, Ly=6.5, H=1.1,
                             mass=5.5e-3 / 2048, speed=20000.0, steps=3000)
    a = _solver(pkg, w, True, monkeypatch)
    o = oracle.model_for(w)
    for _ in range(30):
        a.step(100)
        assert o.step(100) == 0
    fa, fo = a.force_history(), o.force_history()
    da, _, _ = a.state()
    do, _, _ = o.state()
    print(f"\nragged plate vs oracle: peak {fa.max():.3f} vs {fo.max():.3f}, repeats "
          f"{pkg.pdn_get_info(a.ctx)['n_repeats']} vs {o.info()['n_repeats']}")
    assert fo.max() > 0.0
    assert abs(fa.max() - fo.max()) <= 5e-3 * fo.max()
    assert pkg.pdn_get_info(a.ctx)["n_repeats"] == o.info()["n_repeats"]
    assert np.abs(da - do).max() <= 5e-3 * np.abs(do).max()
    a.close()
    o.close()


def test_full_size_plates_plan_a_sweep(pkg, monkeypatch):
    """Asked for (PDN_SWEEP=1), the 128x192x16 plate gets 8 x 4 tiles, the
    400x600x32 plate 16 x 8 tiles (the first shape whose tiles give each of
    the 152 SMs eight blocks)."""
    monkeypatch.setenv("PDN_SWEEP", "1")
    for w, tile in ((pi.damage_fp32_plate(), 3), (pi.large_fp32_plate(), 1)):
        c = pkg.pdn_init_mesh(w.plate, w.material, precision=pkg.PDN_FP32_FORCE)
        info = pkg.pdn_get_info(c)
        assert info["sweep"] == tile
        c.close()
