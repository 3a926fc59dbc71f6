"""The AS4/8552 drop-weight coupon of Sec. 3.2 on the CUDA path: the
Tchamwa-Wielgosz predictor with phi = 1.033 (Sec. 2.2.1), gravity on plate
and striker, the frame and clamp supports and the Table 1 material, against
the FP64 oracle through the C ABI.

Tolerances as in test_gpu_parity: FP64 element mode, contact set identical
and displacements within 1e-9 of the largest; FP32 element mode, peak contact
force within 0.5 % of the oracle's.
"""
import numpy as np
import pytest

import oracle
import pdn_inputs as pi

pytestmark = pytest.mark.gpu

F64_TOL = 1e-9
F32_DISP_TOL = 1e-4
F32_PEAK_TOL = 5e-3


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _run_both(pkg, w, chunks, every, state=None, check_contact=True):
    g = pkg.Solver(w)
    o = oracle.model_for(w)
    if state is not None:
        pkg.pdn_set_state(g.ctx, *state)
        o.set_state(*state)
    for _ in range(chunks):
        g.step(every)
        assert o.step(every) == 0
        if check_contact:
            ag, _ = pkg.pdn_get_contact(g.ctx)
            ao, _ = o.active()
            assert np.array_equal(ag, ao), "contact set differs"
    return g, o


def test_free_fall_follows_the_tw_closed_form(pkg):
    """A free plate falling under gravity (no strain) with phi = 1.033:
    v^n = n dt g and d^n = dt^2 g (n(n-1)/2 + n phi) on the device, the
    first step included (a^0 from the momentum equation at step 0)."""
    plate = pi.make_plate(4.0, 4.0, 1.0, 2, 2, [0.0, 90.0], 1, cohesive=True, clamp="none")
    mat = pi.material_as4_8552(t_ply=0.5, spread=0.0)
    g = -9810.0
    ctx = pkg.pdn_init_mesh(plate, mat, precision=pkg.PDN_FP64, phi=1.033, gravity=(0.0, 0.0, g))
    pkg.pdn_set_impactor(ctx, 1.0, 1e-3, (2.0, 2.0, 1e6), (0.0, 0.0, -1.0))
    n = 60
    pkg.pdn_step(ctx, n)
    dt = pkg.pdn_get_info(ctx)["dt"]
    d, v, imp = pkg.pdn_get_state(ctx)
    assert np.allclose(v[2], n * dt * g, rtol=1e-12, atol=0.0)
    assert np.allclose(d[2], dt * dt * g * (n * (n - 1) / 2.0 + n * 1.033), rtol=1e-11, atol=0.0)
    assert np.abs(d[:2]).max() < 1e-8 * np.abs(d[2]).max()
    # the striker falls freely too (RK4 is exact for constant acceleration)
    assert imp["velocity"][2] == pytest.approx(-1.0 + n * dt * g, rel=1e-12)
    ctx.close()


def test_reduced_coupon_fp64_impact_matches_oracle(pkg):
    """The cut-down coupon (40x28 elements of 0.725 mm, 8 cluster layers,
    frame window and clamps) from rest: 1600 steps of FP64 impact with
    damage onset under the striker; contact set identical every 100 steps,
    displacements and the force history to FP64 round-off."""
    w = pi.reduced_as4_frame_plate(fp64=True)
    g, o = _run_both(pkg, w, 16, 100)
    dg, vg, _ = g.state()
    do, vo, _ = o.state()
    assert _rel(dg, do) < F64_TOL
    assert _rel(vg, vo) < 1e-7
    fg, fo = g.force_history(), o.force_history()
    assert len(fg) == len(fo) == 1600
    assert fo.max() > 300.0
    assert np.abs(fg - fo).max() < 1e-8 * fo.max()
    hist, _ = o.history()
    assert (hist[:, :, :4] > 1.0).any(), "case must damage"
    # supports: the window edge holds z only, the clamps hold every component
    fixed = w.plate.fixed
    assert (dg[2, fixed == 4] == 0.0).all() and (dg[:, fixed == 7] == 0.0).all()
    assert np.abs(dg[:2, fixed == 4]).max() > 0.0
    g.close()


def test_reduced_coupon_fp64_interfaces_from_seeded_state(pkg):
    """A damaging seeded state (dimple + per-node jitter) on the cut-down
    coupon: intralaminar and interface damage with the AS4/8552 constants;
    FP64 GPU == oracle, interface damage field included."""
    w = pi.reduced_as4_frame_plate(fp64=True)
    Lx, Ly, H = w.plate.dims
    st = pi.seeded_state(w.plate, 3, amp=0.03, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.2, 2.0))
    g, o = _run_both(pkg, w, 4, 15, state=st)
    dg, _, _ = g.state()
    do, _, _ = o.state()
    assert _rel(dg, do) < F64_TOL
    hist, rD = o.history()
    assert (hist[:, :, :4] > 1.0).any() and (rD > 0).any(), "case must damage plies and interfaces"
    got = pkg.pdn_damage_field(g.ctx, "DCOH")
    assert np.abs(got - rD.max(axis=1)).max() < 1e-6
    g.close()


def test_reduced_coupon_fp32_peak_force(pkg):
    """FP32 element arithmetic against the FP64 oracle on the cut-down
    coupon through the force peak (2400 steps): peak within 0.5 %."""
    w = pi.reduced_as4_frame_plate(fp64=False, steps=2400)
    g, o = _run_both(pkg, w, 8, 300, check_contact=False)
    fg, fo = g.force_history(), o.force_history()
    k = int(np.argmax(fo))
    assert 0 < k < len(fo) - 50, "the run must pass the peak"
    assert abs(fg.max() - fo.max()) <= F32_PEAK_TOL * fo.max()
    dg, _, _ = g.state()
    do, _, _ = o.state()
    assert _rel(dg, do) < 1e-2
    g.close()


def test_full_size_coupon_steps(pkg):
    """The full coupon (150x100 mm, 207x138x8 hex8, 228,528 hexes and
    171,396 interface elements) from a damaging seeded state: 3 FP32 steps
    against the oracle at every node."""
    w = pi.as4_frame_plate()
    Lx, Ly, H = w.plate.dims
    st = pi.seeded_state(w.plate, 5, amp=0.05, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.15, 4.0))
    g, o = _run_both(pkg, w, 1, 3, state=st, check_contact=False)
    dg, vg, _ = g.state()
    do, vo, _ = o.state()
    assert _rel(dg, do) < F32_DISP_TOL
    assert _rel(vg, vo) < 1e-3
    g.close()


def test_batch_of_coupons_with_gravity_matches_oracle(pkg):
    """Three cut-down coupons of different sizes and seeds in one batch with
    phi = 1.033 and gravity (options common to the batch): every plate
    follows the FP64 oracle (contact set every 150 steps, displacements)."""
    ws = [pi.reduced_as4_frame_plate(nx=nx, ny=ny, fp64=True, seed=s)
          for nx, ny, s in ((24, 18, 1), (32, 22, 2), (40, 28, 3))]
    b = pkg.pdn_batch_init([w.plate for w in ws], [w.material for w in ws], precision=pkg.PDN_FP64,
                           damage_on=True, plasticity_on=True, dt_safety=0.5, phi=1.033,
                           gravity=(0.0, 0.0, -9810.0))
    for c, w in zip(b.plates, ws):
        pkg.pdn_set_impactor(c, *w.impactor())
    orc = [oracle.model_for(w) for w in ws]
    for _ in range(4):
        pkg.pdn_batch_step(b, 150)
        for c, o in zip(b.plates, orc):
            assert o.step(150) == 0
            ag, _ = pkg.pdn_get_contact(c)
            ao, _ = o.active()
            assert np.array_equal(ag, ao), "contact set differs"
    for c, o in zip(b.plates, orc):
        dg, _, _ = pkg.pdn_get_state(c)
        do, _, _ = o.state()
        assert _rel(dg, do) < F64_TOL
        assert o.force_history().max() > 0.0
    b.close()


@pytest.mark.parametrize("fp64,variant", [(True, None), (False, "0"), (False, "4")])
def test_local_repeat_equals_full_repeat(pkg, monkeypatch, fp64, variant):
    """Repetitions of a step after releases (Algorithm 2) evaluate only the
    elements of the released nodes and their nodes; with PDN_FULL_REPEAT=1
    they evaluate everything.  The cut-down coupon through 2000 steps with
    repetitions gives bitwise the same state, contact set, force history and
    damage fields either way (FP64, FP32, and the FP32 kernel that evaluates
    hexes and interfaces in one launch). The element variant is fixed, so
    that both runs execute the same kernels."""
    if variant is not None:
        monkeypatch.setenv("PDN_HEX_VARIANT", variant)
    w = pi.reduced_as4_frame_plate(fp64=fp64)
    runs = []
    for full in ("0", "1"):
        monkeypatch.setenv("PDN_FULL_REPEAT", full)
        g = pkg.Solver(w)
        g.step(2000)
        d, v, imp = g.state()
        act, lam = pkg.pdn_get_contact(g.ctx)
        fields = [pkg.pdn_damage_field(g.ctx, f) for f in ("D1", "D2", "D6", "DCOH")]
        runs.append((d, v, act, lam, g.force_history(), fields, g.info()))
        g.close()
    (d0, v0, a0, l0, f0, k0, i0), (d1, v1, a1, l1, f1, k1, i1) = runs
    assert i0["n_repeats"] == i1["n_repeats"] > 5
    if variant is not None:
        assert i0["hex_variant"] == i1["hex_variant"] == int(variant)
    assert np.array_equal(d0, d1) and np.array_equal(v0, v1)
    assert np.array_equal(a0, a1) and np.array_equal(l0, l1)
    assert np.array_equal(f0, f1)
    for x, y in zip(k0, k1):
        assert np.array_equal(x, y)
