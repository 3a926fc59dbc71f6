"""Interfaces as node pairs (pdn_info.coh_pairs).  Interface elements take
their Newton-Cotes points at the corners (Sec. 2.3.2), and flat interfaces
have the global frame, so the traction at a point depends only on the jump
of the two coincident nodes there and on the point's threshold r_D; every
element around a node pair sees the same jump and, from the undamaged start,
the same history.  The gather then evaluates the cohesive law (Algorithm 5)
once per node and adds each incident element's share in CSR order.

Against interface elements (PDN_COH_PAIRS=0, the interface kernel and its
force slots; element variant 0 on both sides): the same states, contact
force histories, history buffers, energies and interface damage fields, bit
for bit, on seeded damaging states (FP32 and FP64), through an impact with
node release and repetition (Algorithm 2), on the cut-down AS4 coupon with
frame, clamps and gravity, on a plate whose element sizes vary (area
weights per node instead of one weight), and on plates whose node ids are
permuted (partners from the pair table instead of the layered numbering).  The products w tau are rounded
alone on both sides, so the sums agree to the bit unless the compiler
contracts the law's own products differently in the two kernels; the test
prints which and bounds the difference at FP32 rounding."""
import numpy as np
import pytest

import pdn_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _solver(pkg, w, pairs, monkeypatch):
    monkeypatch.setenv("PDN_HEX_VARIANT", "0")
    monkeypatch.setenv("PDN_COH_PAIRS", "1" if pairs else "0")
    s = pkg.Solver(w)
    monkeypatch.delenv("PDN_COH_PAIRS")
    return s


def _graded_plate():
    """A 24x32x8 plate whose columns and rows are graded (x and y each
    mapped by a smooth monotone stretch), so hexes stay axis-aligned boxes and
    interfaces flat rectangles while their areas all differ."""
    w = pi.damage_fp32_plate(nx=24, ny=32, plies=8, Lx=12.0, Ly=16.0, H=2.2, steps=120)
    Lx, Ly, _ = w.plate.dims
    x, y = w.plate.X[0].copy(), w.plate.X[1].copy()
    w.plate.X[0] = x + 0.06 * Lx / (2 * np.pi) * np.sin(2 * np.pi * x / Lx)
    w.plate.X[1] = y - 0.05 * Ly / (2 * np.pi) * np.sin(2 * np.pi * y / Ly)
    return w


def _renumbered(w, seed=3):
    """The same plate with its node ids permuted at random: interfaces stay
    flat, but the numbering is no longer layered (partners from a table)."""
    import dataclasses
    P = w.plate
    perm = np.random.default_rng(seed).permutation(P.n_nodes)  # new id of old node i
    inv = np.empty_like(perm)
    inv[perm] = np.arange(P.n_nodes)
    plate = dataclasses.replace(P, X=np.ascontiguousarray(P.X[:, inv]), hex=perm[P.hex].astype(np.int32),
                                coh=perm[P.coh].astype(np.int32), fixed=np.ascontiguousarray(P.fixed[inv]),
                                surf=np.sort(perm[P.surf]).astype(np.int32))
    return dataclasses.replace(w, plate=plate)


def _cases():
    out = []
    w = pi.damage_fp32_plate(nx=32, ny=48, plies=8, Lx=12.5, Ly=18.75, H=2.2, steps=120)
    out.append(("seeded_32x48x8_fp32", w, True))
    w = pi.damage_fp32_plate(nx=16, ny=24, plies=8, Lx=12.5, Ly=18.75, H=2.2, steps=60, fp64=True)
    out.append(("seeded_16x24x8_fp64", w, True))
    w = pi.damage_fp32_plate(nx=20, ny=13, plies=4, elems_per_ply=2, Lx=10.0, Ly=6.5, H=1.1,
                             mass=5.5e-3 / 2048, speed=20000.0, steps=3000)
    out.append(("impact_release_20x13x8", w, False))
    out.append(("as4_cut_down_40x28x8_fp32", pi.reduced_as4_frame_plate(fp64=False, steps=2000), False))
    out.append(("graded_24x32x8", _graded_plate(), True))
    w = pi.damage_fp32_plate(nx=20, ny=13, plies=4, elems_per_ply=2, Lx=10.0, Ly=6.5, H=1.1,
                             mass=5.5e-3 / 2048, speed=20000.0, steps=3000)
    out.append(("renumbered_impact_20x13x8", _renumbered(w), False))
    w = pi.damage_fp32_plate(nx=16, ny=24, plies=8, Lx=12.5, Ly=18.75, H=2.2, steps=60)
    out.append(("renumbered_seeded_16x24x8", _renumbered(w), True))
    return out


def _seed(pkg, w, *solvers):
    Lx, Ly, _ = w.plate.dims
    st = pi.seeded_state(w.plate, 7, amp=0.02, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.12, 1.5))
    for s in solvers:
        pkg.pdn_set_state(s.ctx, *st)


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / s if s > 0 else np.abs(a - b).max()


@pytest.mark.parametrize("name,w,seeded", _cases(), ids=[c[0] for c in _cases()])
def test_pairs_equal_interface_elements(pkg, monkeypatch, name, w, seeded):
    a = _solver(pkg, w, True, monkeypatch)
    b = _solver(pkg, w, False, monkeypatch)
    # layered numbering (partner from the node id) unless renumbered
    assert pkg.pdn_get_info(a.ctx)["coh_pairs"] == (1 if name.startswith("renumbered") else 2)
    assert pkg.pdn_get_info(b.ctx)["coh_pairs"] == 0
    if seeded:
        _seed(pkg, w, a, b)
    for _ in range(4):
        a.step(w.steps // 4)
        b.step(w.steps // 4)
        assert np.array_equal(pkg.pdn_get_contact(a.ctx)[0], pkg.pdn_get_contact(b.ctx)[0])
    da, va, ia = a.state()
    db, vb, ib = b.state()
    fa, fb = a.force_history(), b.force_history()
    ha, ra = pkg.pdn_get_history(a.ctx)
    hb, rb = pkg.pdn_get_history(b.ctx)
    ea, eb = pkg.pdn_energies(a.ctx), pkg.pdn_energies(b.ctx)
    ca, cb = pkg.pdn_damage_field(a.ctx, "DCOH"), pkg.pdn_damage_field(b.ctx, "DCOH")
    na, nb = pkg.pdn_get_info(a.ctx)["n_repeats"], pkg.pdn_get_info(b.ctx)["n_repeats"]
    bitwise = (np.array_equal(da, db) and np.array_equal(va, vb) and np.array_equal(fa, fb)
               and np.array_equal(ha, hb) and np.array_equal(ra, rb))
    print(f"\n{name}: bitwise {bitwise}, d {_rel(da, db):.2e}, v {_rel(va, vb):.2e}, "
          f"r_D max {rb.max():.3f}, damaged interface points {(rb > 0).sum()}, "
          f"peak {fb.max() if fb.size else 0.0:.3f} N, repeats {na}/{nb}")
    if seeded:
        assert (rb > 0).any(), "case must damage interfaces"
    if "impact" in name:
        assert nb > 0, "case must release nodes"
    assert na == nb
    assert _rel(da, db) <= 1e-6 and _rel(va, vb) <= 1e-4
    assert np.abs(ra - rb).max() <= 1e-5
    assert _rel(ha, hb) <= 1e-5
    if fb.size:
        assert np.abs(fa - fb).max() <= 1e-5 * np.abs(fb).max()
    assert np.abs(ca - cb).max() <= 1e-5
    assert np.abs(ca - ra.max(axis=0)).max() <= 1e-6
    for k in ("ke_plate", "ke_striker", "stored_hex", "stored_interface"):
        assert ea[k] == pytest.approx(eb[k], rel=1e-5, abs=1e-12)
    a.close()
    b.close()


def test_internal_force_equals_interface_elements(pkg, monkeypatch):
    """pdn_internal_force at a seeded damaging state (no step taken): the
    pair gather's forces against the interface kernel's."""
    w = pi.damage_fp32_plate(nx=32, ny=48, plies=8, Lx=12.5, Ly=18.75, H=2.2, steps=10)
    a = _solver(pkg, w, True, monkeypatch)
    b = _solver(pkg, w, False, monkeypatch)
    _seed(pkg, w, a, b)
    fa, fb = pkg.pdn_internal_force(a.ctx), pkg.pdn_internal_force(b.ctx)
    print(f"\ninternal force: bitwise {np.array_equal(fa, fb)}, rel {_rel(fa, fb):.2e}")
    assert _rel(fa, fb) <= 1e-6
    a.close()
    b.close()


def test_pairs_are_the_default_where_the_mesh_allows(pkg, monkeypatch):
    """Node pairs on the benchmark plates (no column sweep unless asked for)
    and in the plates of a batch (the batched kernel's gather evaluates them
    too); none without interfaces or with PDN_COH_PAIRS=0."""
    monkeypatch.delenv("PDN_SWEEP", raising=False)
    monkeypatch.delenv("PDN_COH_PAIRS", raising=False)
    w = pi.damage_fp32_plate()
    c = pkg.pdn_init_mesh(w.plate, w.material, precision=pkg.PDN_FP32_FORCE)
    info = pkg.pdn_get_info(c)
    assert info["coh_pairs"] == 2 and info["sweep"] == 0
    c.close()
    w = pi.plain_fp64_plate(nx=8, ny=8)
    c = pkg.pdn_init_mesh(w.plate, w.material, precision=pkg.PDN_FP64)
    assert pkg.pdn_get_info(c)["coh_pairs"] == 0
    c.close()
    w = pi.damage_fp32_plate(nx=8, ny=12, plies=4, Lx=4.0, Ly=6.0, H=1.1)
    bt = pkg.pdn_batch_init([w.plate, w.plate], [w.material, w.material])
    for p in range(2):
        assert pkg.pdn_get_info(pkg.pdn_batch_plate(bt, p))["coh_pairs"] == 2
    bt.close()
    monkeypatch.setenv("PDN_COH_PAIRS", "0")
    c = pkg.pdn_init_mesh(w.plate, w.material, precision=pkg.PDN_FP32_FORCE)
    assert pkg.pdn_get_info(c)["coh_pairs"] == 0
    c.close()

