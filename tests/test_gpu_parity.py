"""CUDA path against the FP64 oracle, through the C ABI.

Tolerances:
  * FP64 element mode: contact set identical at every checked step; nodal
    displacements within 1e-9 of the largest displacement (the two sides
    differ only in floating-point operation order and FMA contraction).
  * FP32 element mode (forces, damage, interface law in FP32; integration,
    striker, gap test in FP64): peak contact force within 0.5 % and nodal
    displacements within 1e-4 of the largest displacement.
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


def _run_both(pkg, w, chunks, every, precision=None, state=None, check_contact=True, **okw):
    g = pkg.Solver(w, precision=precision)
    o = oracle.model_for(w, **okw)
    if state is not None:
        pkg.pdn_set_state(g.ctx, *state)
        o.set_state(*state)
    for _ in range(chunks):
        g.step(every)
        assert o.step(every) == 0
        if check_contact:
            ag, lg = pkg.pdn_get_contact(g.ctx)
            ao, lo = o.active()
            assert np.array_equal(ag, ao), "contact set differs"
    return g, o


def test_plain_fp64_plate_full_run(pkg):
    """The 40x40x4 mm [0/90]2s plate, FP64, 2000 steps: identical contact set
    every 50 steps, displacements and force history to FP64 round-off."""
    w = pi.plain_fp64_plate()
    g, o = _run_both(pkg, w, 40, 50)
    dg, vg, ig = g.state()
    do, vo, ao = o.state()
    assert _rel(dg, do) < F64_TOL
    assert _rel(vg, vo) < 1e-7
    fg, fo = g.force_history(), o.force_history()
    assert len(fg) == len(fo) == 2000
    assert np.abs(fg - fo).max() < 1e-8 * fo.max()
    assert fo.max() > 300.0
    info, oi = g.info(), o.info()
    assert info["step"] == 2000
    assert info["dt"] == pytest.approx(oi["dt"], rel=1e-14)
    assert ig["centre"] == pytest.approx(o.impactor()["centre"], rel=1e-14)


def _damage_plate(nx=16, ny=24, plies=8, fp64=True):
    return pi.damage_fp32_plate(nx=nx, ny=ny, plies=plies, Lx=12.5, Ly=18.75, H=2.2, fp64=fp64)


def _damaging_state(w, seed=7):
    Lx, Ly, H = w.plate.dims
    return pi.seeded_state(w.plate, seed, amp=0.02, vamp=300.0,
                           dimple=(0.5 * Lx, 0.5 * Ly, 0.12, 1.5))


def test_fp64_damage_and_interfaces_from_seeded_state(pkg):
    """Damaging seeded state (dimple + jitter): intralaminar damage,
    plasticity and interface damage all active; FP64 GPU == oracle."""
    w = _damage_plate(fp64=True)
    st = _damaging_state(w)
    g, o = _run_both(pkg, w, 6, 10, state=st)
    dg, vg, _ = g.state()
    do, vo, _ = o.state()
    assert _rel(dg, do) < F64_TOL
    hist, rD = o.history()
    assert (hist[:, :, :4] > 1.0).any(), "case must damage"
    assert (rD > 0).any(), "case must damage interfaces"
    assert (hist[:, :, 6] > 0).any(), "case must yield"
    # damage fields: element max over points of the oracle's history
    lc, sf = o.lc(), o.strength_factors()
    exp = np.array([[oracle.damage_of_history(w.material, lc[e], sf[e], hist[e, gp]) for gp in range(8)]
                    for e in range(w.plate.n_hex)])  # [n_hex, 8, (D1, D2, D6)]
    for k, name in enumerate(("D1", "D2", "D6")):
        got = pkg.pdn_damage_field(g.ctx, name)
        assert np.abs(got - exp[:, :, k].max(axis=1)).max() < 1e-6
    got = pkg.pdn_damage_field(g.ctx, "DCOH")
    assert np.abs(got - rD.max(axis=1)).max() < 1e-6
    # equivalent plastic shear strain: element maximum of the last history field
    got = pkg.pdn_damage_field(g.ctx, "PLASTIC")
    want = hist[:, :, 6].max(axis=1)
    assert want.max() > 0.0
    assert np.abs(got - want).max() <= 1e-6 * want.max()
    # the device-pointer output gives the same floats
    import torch
    dev = torch.zeros(w.plate.n_hex, dtype=torch.float32, device="cuda")
    pkg.pdn_damage_field(g.ctx, "D2", out=dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), pkg.pdn_damage_field(g.ctx, "D2"))


def test_fp32_damage_from_seeded_state(pkg):
    w = _damage_plate(fp64=False)
    st = _damaging_state(w)
    g, o = _run_both(pkg, w, 6, 10, state=st, check_contact=False)
    dg, _, _ = g.state()
    do, _, _ = o.state()
    assert _rel(dg, do) < F32_DISP_TOL


def _distorted(w, amp=0.06, seed=2):
    """The plate with its node columns moved in-plane by seeded amounts (the
    coincident interface layers move together): the hexes are no longer
    boxes and the interfaces no longer rectangles, so the general element
    kernels run instead of the box and flat-rectangle ones."""
    import dataclasses
    p = w.plate
    rng = np.random.default_rng(seed)
    _, col = np.unique(np.round(p.X[:2].T, 9), axis=0, return_inverse=True)
    shift = rng.uniform(-amp, amp, size=(col.max() + 1, 2))
    X = p.X.copy()
    X[:2] += shift[col.ravel()].T
    q = dataclasses.replace(p, X=X)
    return dataclasses.replace(w, plate=q)


@pytest.mark.parametrize("fp64", [True, False])
def test_distorted_mesh_matches_oracle(pkg, fp64):
    """General hex8 and interface kernels on a distorted plate from a
    damaging seeded state, against the oracle (FP64: contact set and 1e-9;
    FP32: 1e-4)."""
    w = _distorted(_damage_plate(fp64=fp64))
    st = _damaging_state(w)
    g, o = _run_both(pkg, w, 6, 10, state=st, check_contact=fp64)
    dg, _, _ = g.state()
    do, _, _ = o.state()
    assert _rel(dg, do) < (F64_TOL if fp64 else F32_DISP_TOL)
    hist, rD = o.history()
    assert (hist[:, :, :4] > 1.0).any() and (rD > 0).any()


def test_csr_slots_when_a_node_has_more_than_eight_elements(pkg):
    """Four hexes appended a second time (a doubled element: the same
    physics for the device and the oracle) give their nodes more than eight
    incident elements, so the element forces use CSR positions instead of
    eight slots per node; FP64 stepping from a damaging seeded state against
    the oracle."""
    import dataclasses
    w = _damage_plate(fp64=True)
    p = w.plate
    extra = np.arange(4) + p.n_hex // 2
    q = dataclasses.replace(p, hex=np.concatenate([p.hex, p.hex[extra]]),
                            ply_of_hex=np.concatenate([p.ply_of_hex, p.ply_of_hex[extra]]))
    w = dataclasses.replace(w, plate=q)
    deg = np.bincount(np.concatenate([q.hex.ravel(), q.coh.ravel()]), minlength=q.n_nodes)
    assert deg.max() > 8
    st = _damaging_state(w)
    g, o = _run_both(pkg, w, 4, 10, state=st)
    dg, _, _ = g.state()
    do, _, _ = o.state()
    assert _rel(dg, do) < F64_TOL


def test_profiled_steps_are_the_same_steps(pkg):
    """pdn_profile_kernels advances real steps, launching each kernel on its
    own between CUDA events (no graph, the interface kernel on the same
    stream): from the same damaging state, 30 stepped + 30 profiled steps end
    bitwise where 60 stepped steps end (FP64: no tuned variant involved), and
    every kernel reports a positive mean time and at least one launch per
    profiled step."""
    w = _damage_plate(fp64=True)
    st = _damaging_state(w)
    a, b = pkg.Solver(w), pkg.Solver(w)
    for g in (a, b):
        pkg.pdn_set_state(g.ctx, *st)
    a.step(60)
    b.step(30)
    prof = pkg.pdn_profile_kernels(b.ctx, 30)
    (da, va, _), (db, vb, _) = a.state(), b.state()
    assert np.array_equal(da, db) and np.array_equal(va, vb)
    assert np.array_equal(a.force_history(), b.force_history())
    assert a.info()["step"] == b.info()["step"]
    for k in pkg.KERNELS:
        ms, n = prof[k]
        assert n >= 30 and ms > 0.0, (k, ms, n)
    a.close()
    b.close()


def test_internal_force_matches_oracle(pkg):
    # FP32: nodal forces are sums of element contributions that largely cancel,
    # so the FP32 error relative to the largest nodal force is ~1e-5..1e-4
    for fp64, tol in ((True, 1e-10), (False, 1e-4)):
        w = _damage_plate(fp64=fp64)
        st = _damaging_state(w, seed=3)
        g = pkg.Solver(w)
        o = oracle.model_for(w)
        pkg.pdn_set_state(g.ctx, *st)
        o.set_state(*st)
        fg = pkg.pdn_internal_force(g.ctx)
        fo = o.internal_force()
        assert _rel(fg, fo) < tol


def test_fp32_impact_peak_force(pkg):
    """Reduced plate with the damage/interface physics of the 100x150 mm
    workload (same element size, layup rule and striker), FP32 element
    arithmetic against the FP64 oracle: peak contact force within 0.5 % and
    displacements within 1e-4."""
    w = pi.damage_fp32_plate(nx=32, ny=48, Lx=25.0, Ly=37.5, H=4.4, mass=5.5e-3 / 16, steps=3000)
    g, o = _run_both(pkg, w, 30, 100, check_contact=False)
    fg, fo = g.force_history(), o.force_history()
    assert fo.max() > 0.0
    assert abs(fg.max() - fo.max()) <= F32_PEAK_TOL * fo.max()
    dg, _, _ = g.state()
    do, _, _ = o.state()
    assert _rel(dg, do) < F32_DISP_TOL


def test_release_and_repeat_matches_oracle(pkg):
    """Rebound of a light striker: adhesive nodes are released and the step
    repeated on the device exactly as in the oracle (FP64)."""
    plate = pi.make_plate(8.0, 8.0, 0.5, 16, 16, [0.0, 90.0], 1, cohesive=False)
    mat = pi.material_im7_like_config(t_ply=0.25, spread=0.0)
    wl = pi.Workload("rebound", plate, mat, True, False, False, 2.0, 2e-6, 3000.0, 1e-4, 0.5, 0)
    g = pkg.Solver(wl)
    o = oracle.model_for(wl)
    for _ in range(90):
        g.step(100)
        assert o.step(100) == 0
        assert np.array_equal(pkg.pdn_get_contact(g.ctx)[0], o.active()[0])
    assert g.info()["n_repeats"] == o.info()["n_repeats"] > 0
    assert g.state()[2]["velocity"][2] == pytest.approx(o.impactor()["velocity"][2], rel=1e-9)


def test_deterministic(pkg, monkeypatch):
    """Two runs of the same launch configuration give bitwise the same state
    (the element-kernel variant is fixed: the autotuner may pick variants
    that contract multiply-adds differently)."""
    monkeypatch.setenv("PDN_HEX_VARIANT", "0")
    w = _damage_plate(fp64=False)
    st = _damaging_state(w)
    out = []
    for _ in range(2):
        g = pkg.Solver(w)
        pkg.pdn_set_state(g.ctx, *st)
        g.step(37)
        d, v, imp = g.state()
        out.append((d, v, g.force_history(), pkg.pdn_damage_field(g.ctx, "D2")))
        g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_full_size_workload_steps(pkg):
    """The 100x150x4.4 mm, 128x192x16 plate (393,216 hexes, the benchmark's
    launch configuration) from a damaging seeded state: 3 steps against the
    oracle at every node."""
    w = pi.damage_fp32_plate()
    Lx, Ly, H = w.plate.dims
    st = pi.seeded_state(w.plate, 5, amp=0.05, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.15, 4.0))
    g, o = _run_both(pkg, w, 1, 3, state=st, check_contact=False)
    dg, vg, _ = g.state()
    do, vo, _ = o.state()
    assert _rel(dg, do) < F32_DISP_TOL
    assert _rel(vg, vo) < 1e-3


@pytest.mark.slow
def test_large_mesh_internal_force(pkg):
    """The 400x600x32 refinement (7.68M hexes): internal force of a seeded
    damaging state at every node against the oracle."""
    w = pi.large_fp32_plate()
    Lx, Ly, H = w.plate.dims
    st = pi.seeded_state(w.plate, 9, amp=0.05, vamp=0.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.1, 4.0))
    g = pkg.Solver(w)
    pkg.pdn_set_state(g.ctx, *st)
    fg = pkg.pdn_internal_force(g.ctx)
    g.close()
    o = oracle.model_for(w)
    o.set_state(*st)
    fo = o.internal_force()
    assert _rel(fg, fo) < 1e-4


# ---------------------------------------------------------------------------
# Edge cases and failure reporting (host-side injection, no GPU fault)

def test_zero_steps_and_no_surface(pkg):
    plate = pi.make_plate(4.0, 4.0, 1.0, 3, 3, [0.0, 90.0], 1, cohesive=True)
    plate.surf = plate.surf[:0]
    mat = pi.material_im7_like_config(t_ply=0.5)
    ctx = pkg.pdn_init_mesh(plate, mat, precision=pkg.PDN_FP64, damage_on=False)
    pkg.pdn_set_impactor(ctx, 1.0, 1e-3, (2.0, 2.0, 1.5), (0.0, 0.0, -100.0))
    pkg.pdn_step(ctx, 0)
    assert pkg.pdn_get_info(ctx)["step"] == 0
    pkg.pdn_step(ctx, 5)
    assert pkg.pdn_get_info(ctx)["step"] == 5
    assert pkg.pdn_get_contact(ctx)[0].size == 0


def test_ragged_step_counts_match_single_call(pkg):
    w = _damage_plate(fp64=True)
    st = _damaging_state(w)
    a = pkg.Solver(w)
    pkg.pdn_set_state(a.ctx, *st)
    a.step(71)
    b = pkg.Solver(w)
    pkg.pdn_set_state(b.ctx, *st)
    for n in (1, 32, 5, 33):
        b.step(n)
    assert np.array_equal(a.state()[0], b.state()[0])


def test_invalid_arguments(pkg):
    plate = pi.make_plate(4.0, 4.0, 1.0, 2, 2, [0.0], 1, cohesive=False)
    mat = pi.material_im7_like_config(t_ply=1.0)
    bad = pi.make_plate(4.0, 4.0, 1.0, 2, 2, [0.0], 1, cohesive=False)
    bad.hex = bad.hex.copy()
    bad.hex[0, 0] = 10 ** 6
    with pytest.raises(pkg.PdnError) as ei:
        pkg.pdn_init_mesh(bad, mat, damage_on=False)
    assert ei.value.code == -1
    dup = pi.make_plate(4.0, 4.0, 1.0, 2, 2, [0.0], 1, cohesive=False)
    dup.surf = np.concatenate([dup.surf, dup.surf[:1]])
    with pytest.raises(pkg.PdnError):
        pkg.pdn_init_mesh(dup, mat, damage_on=False)
    # 1 mm elements, past the compressive matrix law's snap-back length, are
    # accepted (the law drops to zero stress at onset there); the learned law
    # is refused at that length
    pkg.pdn_init_mesh(plate, mat, damage_on=True).close()
    with pytest.raises(pkg.PdnError) as ei:
        pkg.pdn_sur_create(mat, 1.0)
    assert ei.value.code == -7
    ctx = pkg.pdn_init_mesh(plate, mat, damage_on=False)
    with pytest.raises(pkg.PdnError) as ei:
        pkg.pdn_step(ctx, 1)  # no striker yet
    assert ei.value.code == -8
    with pytest.raises(pkg.PdnError):
        pkg.pdn_damage_field(ctx, 99)


def test_nonfinite_state_is_reported_and_sticky(pkg):
    w = _damage_plate(fp64=False)
    g = pkg.Solver(w)
    d, v = _damaging_state(w)
    d[2, d.shape[1] // 2] = np.nan
    with pytest.raises(pkg.PdnError) as ei:
        pkg.pdn_set_state(g.ctx, d, v)
    assert ei.value.code == -4
    with pytest.raises(pkg.PdnError) as ei:
        g.step(1)
    assert ei.value.code == -4


def test_release_limit_is_reported(pkg):
    """With repetitions disabled, the first adhesive node ends the run with
    PDN_E_RELEASE_LIMIT (host-checked status, no device fault)."""
    plate = pi.make_plate(8.0, 8.0, 0.5, 16, 16, [0.0, 90.0], 1, cohesive=False)
    mat = pi.material_im7_like_config(t_ply=0.25, spread=0.0)
    wl = pi.Workload("rebound", plate, mat, True, False, False, 2.0, 2e-6, 3000.0, 1e-4, 0.5, 0)
    g = pkg.Solver(wl, max_release_iters=-1)
    with pytest.raises(pkg.PdnError) as ei:
        for _ in range(100):
            g.step(100)
    assert ei.value.code == -5
