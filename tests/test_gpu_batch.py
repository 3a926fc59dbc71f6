"""Batched persistent launch (include/pdn_batch.h) through the C ABI.

A batch steps independent plates together; every plate must follow the FP64
oracle exactly as a plate stepped alone does (contact set identical,
displacements to 1e-9 of the largest).  A plate stepped in a batch follows
the same plate stepped alone by pdn_step to rounding: both run the same
per-item source code and fixed reduction orders, but the compiler may
contract multiply-adds differently in different kernels.  Repeated runs of
one schedule are bitwise identical.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import pdn_inputs as pi

pytestmark = pytest.mark.gpu

F64_TOL = 1e-9


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _cases(n, seed, hex_min, hex_max, fp64, gap=0.001):
    """Small seeded batch cases with a small initial gap, so that contact
    starts within the first few hundred steps."""
    return [dataclasses.replace(w, gap=gap) for w in
            pi.batch_plates(n=n, seed=seed, hex_min=hex_min, hex_max=hex_max, fp64=fp64)]


def _batch(pkg, ws, fp64):
    b = pkg.pdn_batch_init([w.plate for w in ws], [w.material for w in ws],
                           precision=pkg.PDN_FP64 if fp64 else pkg.PDN_FP32_FORCE,
                           damage_on=True, plasticity_on=True, dt_safety=0.5)
    for c, w in zip(b.plates, ws):
        pkg.pdn_set_impactor(c, *w.impactor())
    return b


@pytest.mark.parametrize("schedule", ["0", "1"])
def test_batch_fp64_matches_oracle(pkg, schedule, monkeypatch):
    """Three FP64 plates of different sizes and layups: the contact set of
    every plate equals the oracle's after every chunk, displacements and
    the force history agree to FP64 round-off (both schedules)."""
    monkeypatch.setenv("PDN_BATCH_SCHEDULE", schedule)
    ws = _cases(3, 11, 1500, 5000, fp64=True)
    b = _batch(pkg, ws, True)
    orc = [oracle.model_for(w) for w in ws]
    for _ in range(4):
        pkg.pdn_batch_step(b, 150)
        for c, o in zip(b.plates, orc):
            assert o.step(150) == 0
            ag, _ = pkg.pdn_get_contact(c)
            ao, _ = o.active()
            assert np.array_equal(ag, ao), "contact set differs"
    touched = 0
    for c, o in zip(b.plates, orc):
        dg, vg, ig = pkg.pdn_get_state(c)
        do, vo, io = o.state()
        assert _rel(dg, do) < F64_TOL
        fg = pkg.pdn_contact_force(c)[2]
        fo = o.force_history()
        assert len(fg) == len(fo) == 600
        scale = max(np.abs(fo).max(), 1e-300)
        assert np.abs(fg - fo).max() / scale < 1e-8
        touched += int(np.abs(fo).max() > 0)
    assert touched >= 2, "the cases should reach contact"
    info = pkg.pdn_batch_get_info(b)
    assert info["tuned"] == 1 and info["status"] == 0
    assert info["passes"] >= 600
    b.close()


@pytest.mark.parametrize("schedule", ["0", "1"])
def test_batch_equals_plates_stepped_alone(pkg, schedule, monkeypatch):
    """FP32 force mode with damage and interfaces: four plates stepped in one
    batch give the same displacements, contact sets and force histories as
    each plate stepped alone, with either schedule (grid barriers, dataflow)."""
    monkeypatch.setenv("PDN_BATCH_SCHEDULE", schedule)
    ws = _cases(4, 5, 2000, 20000, fp64=False)
    b = _batch(pkg, ws, False)
    pkg.pdn_batch_step(b, 700)
    assert pkg.pdn_batch_get_info(b)["dataflow"] == int(schedule)
    for c, w in zip(b.plates, ws):
        s = pkg.Solver(dataclasses.replace(w), precision=pkg.PDN_FP32_FORCE)
        s.step(700)
        d1, v1, i1 = pkg.pdn_get_state(c)
        d2, v2, i2 = s.state()
        assert _rel(d1, d2) < 1e-5, _rel(d1, d2)
        # velocities carry the high-frequency part of the rounding-level
        # differences between the two kernel instantiations, grown through
        # the damage steps
        assert _rel(v1, v2) < 1e-3, _rel(v1, v2)
        a1, _ = pkg.pdn_get_contact(c)
        a2, _ = pkg.pdn_get_contact(s.ctx)
        assert np.array_equal(a1, a2)
        f1 = pkg.pdn_contact_force(c)[2]
        f2 = s.force_history()
        assert np.abs(f1 - f2).max() <= 1e-5 * max(np.abs(f2).max(), 1e-300)
        for field in ("D2", "DCOH"):
            assert np.allclose(pkg.pdn_damage_field(c, field), pkg.pdn_damage_field(s.ctx, field), atol=1e-5)
        s.close()
    b.close()


@pytest.mark.parametrize("schedule", ["0,0", "0,1", "1,0", "1,1"])
def test_batch_is_deterministic(pkg, schedule, monkeypatch):
    """Two batches with the same schedule and register variant give bitwise
    identical states and force histories (no race between tiles)."""
    monkeypatch.setenv("PDN_BATCH_SCHEDULE", schedule)
    ws = _cases(3, 5, 2000, 20000, fp64=False)
    outs = []
    for _ in range(2):
        b = _batch(pkg, ws, False)
        pkg.pdn_batch_step(b, 700)
        info = pkg.pdn_batch_get_info(b)
        assert (info["dataflow"], info["reg_variant"]) == tuple(int(x) for x in schedule.split(","))
        outs.append([(pkg.pdn_get_state(c)[0], pkg.pdn_contact_force(c)[2]) for c in b.plates])
        b.close()
    for (d1, f1), (d2, f2) in zip(*outs):
        assert np.array_equal(d1, d2) and np.array_equal(f1, f2)


def test_batch_ragged_steps_and_info(pkg):
    ws = _cases(3, 2, 1000, 4000, fp64=False)
    b = _batch(pkg, ws, False)
    pkg.pdn_batch_step(b, 37)
    pkg.pdn_batch_step(b, 0)
    pkg.pdn_batch_step(b, 50)
    for c in b.plates:
        assert pkg.pdn_get_info(c)["step"] == 87
    info = pkg.pdn_batch_get_info(b)
    assert info["n_plates"] == 3 and info["tuned"] == 1
    assert info["n_candidates"] >= 2 and len(info["candidates"]) == info["n_candidates"]
    assert info["grid"] > 0 and info["blocks_per_sm"] >= 1
    assert info["n_tiles"][3] == 3  # one tail tile per plate
    assert info["passes"] >= 87 and info["launches"] >= 2
    # a plate of the batch can still be stepped alone
    pkg.pdn_step(b.plates[0], 5)
    assert pkg.pdn_get_info(b.plates[0])["step"] == 92
    pkg.pdn_batch_step(b, 3)
    assert [pkg.pdn_get_info(c)["step"] for c in b.plates] == [95, 90, 90]
    b.close()


@pytest.mark.parametrize("schedule", ["0", "1"])
def test_batch_plates_without_surface_or_interfaces(pkg, schedule, monkeypatch):
    """A plate without contact surface (no contact tiles: its element tiles
    depend directly on its previous tail) and a plate without interface
    elements, next to a regular plate, in both schedules: each follows the
    same plate stepped alone."""
    monkeypatch.setenv("PDN_BATCH_SCHEDULE", schedule)
    base = _cases(3, 8, 2000, 6000, fp64=False)
    w_nosurf = dataclasses.replace(base[0], plate=dataclasses.replace(base[0].plate,
                                                                      surf=np.zeros(0, dtype=np.int32)))
    p1 = base[1].plate
    lay = list(p1.ply_angle_deg)
    Lx, Ly, H = p1.dims
    nx, ny, _ = p1.grid
    w_nocoh = dataclasses.replace(base[1], plate=pi.make_plate(Lx, Ly, H, nx, ny, lay, 1, cohesive=False))
    ws = [w_nosurf, w_nocoh, base[2]]
    assert ws[0].plate.n_surf == 0 and ws[1].plate.n_coh == 0 and ws[2].plate.n_coh > 0
    b = _batch(pkg, ws, False)
    pkg.pdn_batch_step(b, 400)
    for c, w in zip(b.plates, ws):
        s = pkg.Solver(w, precision=pkg.PDN_FP32_FORCE)
        s.step(400)
        assert pkg.pdn_get_info(c)["step"] == 400
        d1, d2 = pkg.pdn_get_state(c)[0], s.state()[0]
        assert _rel(d1, d2) < 1e-5
        f1, f2 = pkg.pdn_contact_force(c)[2], s.force_history()
        assert np.abs(f1 - f2).max() <= 1e-5 * max(np.abs(f2).max(), 1e-300)
        s.close()
    assert np.abs(pkg.pdn_contact_force(b.plates[0])[2]).max() == 0.0  # no surface, no contact
    assert np.abs(pkg.pdn_contact_force(b.plates[1])[2]).max() > 0.0
    b.close()


def test_batch_requires_every_striker(pkg):
    ws = _cases(2, 3, 1000, 2000, fp64=False)
    b = pkg.pdn_batch_init([w.plate for w in ws], [w.material for w in ws])
    pkg.pdn_set_impactor(b.plates[0], *ws[0].impactor())
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_batch_step(b, 1)
    assert e.value.code == -8 and "plate 1" in str(e.value)
    b.close()


def test_batch_barrier_wait_is_bounded(pkg):
    """A launch in which one block never arrives: the others give up after
    the time limit, the status is PDN_E_TIMEOUT, and the batch goes on
    stepping with unchanged results afterwards."""
    ws = _cases(2, 4, 1000, 3000, fp64=False)
    b = _batch(pkg, ws, False)
    pkg.pdn_batch_step(b, 20)
    d_before = pkg.pdn_get_state(b.plates[0])[0]
    rc = pkg.pdn_batch_test_barrier_timeout(b, 50.0)
    assert rc == -6
    assert np.array_equal(pkg.pdn_get_state(b.plates[0])[0], d_before)
    pkg.pdn_batch_step(b, 30)
    s = pkg.Solver(dataclasses.replace(ws[0]), precision=pkg.PDN_FP32_FORCE)
    s.step(50)
    assert _rel(pkg.pdn_get_state(b.plates[0])[0], s.state()[0]) < 1e-5
    s.close()
    b.close()


def test_batch_full_config_few_steps(pkg):
    """The 64-plate batch (8k-400k hex8 per plate, 6.2M in total): a few
    steps run, every plate advances, and the smallest plates agree with the
    same plates stepped alone."""
    ws = [dataclasses.replace(w, gap=0.0) for w in pi.batch_plates(n=64, seed=0)]
    b = _batch(pkg, ws, False)
    pkg.pdn_batch_step(b, 12)
    steps = [pkg.pdn_get_info(c)["step"] for c in b.plates]
    assert steps == [12] * 64
    order = np.argsort([w.plate.n_hex for w in ws])[:2]
    for k in order:
        s = pkg.Solver(ws[k], precision=pkg.PDN_FP32_FORCE)
        s.step(12)
        assert _rel(pkg.pdn_get_state(b.plates[k])[0], s.state()[0]) < 1e-5
        s.close()
    b.close()
