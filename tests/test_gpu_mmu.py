"""Mesh multiplication on the device (include/pdn_mmu.h; Sec. 2.4, Eq. mmu,
Algorithm 3) against the oracle (oracle/mesh_multiply.py) through the C ABI, up to the
AS4/8552 coupon's full size.

Node numbering, connectivity, plies, constraint bits and the surface list are
integer results: bit-exact.  Coordinates are means of 2, 4 or 8 FP64 values
summed in a stated order: bit-exact as well.  At the coupon's full size the
division is also checked by properties that hold at any size, and the solver
on the refined mesh by a few steps against the FP64 oracle.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import oracle.mesh_multiply as mm
import pdn_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _jittered(p, amp, seed):
    """The plate with its in-plane node positions jittered; coincident
    interface layers stay coincident."""
    rng = np.random.default_rng(seed)
    X = p.X.copy()
    moved = {}
    for j in range(X.shape[1]):
        k = (round(p.X[0, j], 9), round(p.X[1, j], 9))
        if k not in moved:
            moved[k] = rng.uniform(-amp, amp, size=2)
        X[:2, j] += moved[k]
    p.X = X
    return p


CASES = {
    "structured_interfaces": lambda: pi.make_plate(4.0, 6.0, 2.0, 5, 7, [0.0, 90.0, 90.0, 45.0, -45.0], 1),
    "distorted": lambda: _jittered(pi.make_plate(3.0, 2.0, 1.5, 6, 5, [0.0, 45.0, 90.0], 1), 0.08, 3),
    "as4_coupon_cut_down": lambda: pi.reduced_as4_frame_plate(nx=24, ny=18).plate,
    "no_interfaces_no_surface": lambda: _strip(pi.make_plate(2.0, 2.0, 1.0, 3, 2, [0.0, 0.0], 1, cohesive=False)),
}


def _strip(p):
    p.surf = p.surf[:0]
    return p


@pytest.mark.parametrize("case,levels", [("structured_interfaces", 1), ("structured_interfaces", 2),
                                         ("structured_interfaces", 3), ("distorted", 2),
                                         ("as4_coupon_cut_down", 1), ("no_interfaces_no_surface", 2)])
def test_division_equals_oracle_bitwise(pkg, case, levels):
    p = CASES[case]()
    r = pkg.pdn_mesh_multiply(p, levels)
    got = pkg.pdn_refined_get(r)
    info = pkg.pdn_refined_get_info(r)
    r.close()
    X, h, c, ply, fx, sf = mm.multiply(p.X, p.hex, p.coh, p.ply_of_hex, p.fixed, p.surf, levels)
    assert info["levels"] == levels and info["device_ms"] > 0.0
    assert (info["n_nodes"], info["n_hex"], info["n_coh"], info["n_surf"]) == (X.shape[1], len(h), len(c), len(sf))
    assert np.array_equal(got["hex"], h)
    assert np.array_equal(got["coh"], c)
    assert np.array_equal(got["ply_of_hex"], ply)
    assert np.array_equal(got["fixed"], fx)
    assert np.array_equal(got["surf"], sf)
    assert np.array_equal(got["X"], X)  # bitwise: same sums in the same order


def test_zero_levels_and_repeated_calls(pkg):
    p = CASES["structured_interfaces"]()
    r = pkg.pdn_mesh_multiply(p, 0)
    got = pkg.pdn_refined_get(r)
    r.close()
    assert np.array_equal(got["X"], p.X) and np.array_equal(got["hex"], p.hex) and np.array_equal(got["surf"], p.surf)
    a = pkg.pdn_refined_get(pkg.pdn_mesh_multiply(p, 2))
    b = pkg.pdn_refined_get(pkg.pdn_mesh_multiply(p, 2))
    for k in a:
        assert np.array_equal(a[k], b[k])


def test_invalid_meshes_are_rejected(pkg):
    p = CASES["structured_interfaces"]()
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_mesh_multiply(p, 7)
    assert e.value.code == -1
    bad = CASES["structured_interfaces"]()
    bad.hex = bad.hex.copy()
    bad.hex[3, 2] = bad.n_nodes
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_mesh_multiply(bad, 1)
    assert e.value.code == -1
    # an interface whose upper face is not a face of any hex
    bad = CASES["structured_interfaces"]()
    bad.coh = bad.coh.copy()
    bad.coh[0, 6] = bad.coh[0, 0]  # a lower-layer node in the upper face
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_mesh_multiply(bad, 1)
    assert e.value.code == -1 and "interface element 0" in str(e.value)


def _box_volumes(X, hexes):
    lo = X[:, hexes[:, 0]]
    hi = X[:, hexes[:, 6]]
    return np.prod(hi - lo, axis=0)


def test_full_coupon_division_properties(pkg):
    """The AS4/8552 coupon (207x138x8 hex8, 228,528 hexes, 171,396
    interfaces) divided once on the device into the paper's 0.3625 mm mesh:
    the counts of Eq. mmu (edges and faces counted on the host), children at
    the parent's lattice points, interface faces that are faces of child
    hexes, volume kept."""
    p = pi.as4_frame_plate().plate
    r = pkg.pdn_mesh_multiply(p, 1)
    info = pkg.pdn_refined_get_info(r)
    g = pkg.pdn_refined_get(r)
    r.close()
    nh, nc, nn = p.n_hex, p.n_coh, p.n_nodes
    E = np.unique(np.sort(p.hex[:, np.array(mm.HEX_EDGES)], axis=2).reshape(-1, 2), axis=0)
    F = np.unique(np.sort(p.hex[:, np.array(mm.HEX_FACES)], axis=2).reshape(-1, 4), axis=0)
    assert info["n_hex"] == 8 * nh and info["n_coh"] == 4 * nc
    assert (info["n_edges"], info["n_faces"]) == (len(E), len(F))
    assert info["n_nodes"] == nn + len(E) + len(F) + nh
    X, H = g["X"], g["hex"]
    # children of parent e are 8e..8e+7; corner a of child (ci, cj, ck) sits
    # at lattice point (ci + a_x, cj + a_y, ck + a_z) of the parent box
    lo = p.X[:, p.hex[:, 0]]
    hi = p.X[:, p.hex[:, 6]]
    for c in range(8):
        ci, cj, ck = c & 1, (c >> 1) & 1, c >> 2
        for a in (0, 6):
            ox, oy, oz = (np.array(mm._CORNER[a]) // 2 + [ci, cj, ck]) / 2.0
            want = lo + (hi - lo) * np.array([[ox], [oy], [oz]])
            assert np.allclose(X[:, H[c::8, a]], want, rtol=0.0, atol=1e-12)
    assert np.sum(_box_volumes(X, H)) == pytest.approx(np.sum(_box_volumes(p.X, p.hex)), rel=1e-12)
    assert np.array_equal(g["ply_of_hex"], np.repeat(p.ply_of_hex, 8))
    # interfaces: lower and upper faces coincide and are faces of child hexes
    C = g["coh"]
    assert np.array_equal(X[:, C[:, :4]], X[:, C[:, 4:]])
    def rows(a):
        a = np.ascontiguousarray(np.sort(a, axis=1).astype(np.int64))
        return a.view(np.dtype((np.void, a.dtype.itemsize * a.shape[1]))).ravel()

    hf = rows(H[:, np.array(mm.HEX_FACES)].reshape(-1, 4))
    for side in (C[:, :4], C[:, 4:]):
        assert np.isin(rows(side), hf).all()
    # the contact surface stays the top face
    assert np.all(X[2, g["surf"]] == p.dims[2]) and len(g["surf"]) == (2 * 207 + 1) * (2 * 138 + 1)
    # and the whole division equals the oracle's, bit for bit (about 30 s of
    # Python on the host)
    Xo, ho, co, po, fo, so, _ = mm.divide_once(p.X, p.hex, p.coh, p.ply_of_hex, p.fixed, p.surf)
    assert np.array_equal(H, ho) and np.array_equal(C, co) and np.array_equal(g["surf"], so)
    assert np.array_equal(g["fixed"], fo) and np.array_equal(X, Xo)


def test_refined_plate_runs_like_the_direct_fine_plate(pkg):
    """FP64 impact on a plate divided on the device and on the plate built
    directly at twice the resolution: same force history to round-off (the
    numbering differs, the mesh does not)."""
    lay = [0.0, 90.0, 90.0, 0.0]
    coarse = pi.make_plate(8.0, 8.0, 2.0, 6, 6, lay, 1, cohesive=True)
    fine = pi.make_plate(8.0, 8.0, 2.0, 12, 12, lay, 2, cohesive=True)
    mat = pi.material_im7_like_config(t_ply=0.5, spread=0.0)
    r = pkg.pdn_mesh_multiply(coarse, 1)
    a = pkg.pdn_init_refined(r, mat, precision=pkg.PDN_FP64, damage_on=False)
    b = pkg.pdn_init_mesh(fine, mat, precision=pkg.PDN_FP64, damage_on=False)
    for ctx in (a, b):
        pkg.pdn_set_impactor(ctx, 3.0, 5e-4, (4.0, 4.0, 2.0 + 3.0 + 0.001), (0.0, 0.0, -2000.0))
        pkg.pdn_step(ctx, 600)
    fa, fb = pkg.pdn_contact_force(a)[2], pkg.pdn_contact_force(b)[2]
    assert pkg.pdn_get_info(a)["dt"] == pytest.approx(pkg.pdn_get_info(b)["dt"], rel=1e-12)
    assert fb.max() > 0.0
    assert np.abs(fa - fb).max() <= 1e-9 * fb.max()
    a.close()
    b.close()
    r.close()


def test_refined_full_coupon_steps_against_oracle(pkg):
    """The coupon divided once on the device (1,828,224 hexes, 685,584
    interfaces) and handed to the solver: 2 FP32 steps from a damaging seeded
    state against the FP64 oracle on the same divided mesh."""
    w = pi.as4_frame_plate()
    r = pkg.pdn_mesh_multiply(w.plate, 1)
    g = pkg.pdn_refined_get(r)
    fine = pi.Plate(X=g["X"], hex=g["hex"], coh=g["coh"], ply_of_hex=g["ply_of_hex"],
                    ply_of_coh=np.repeat(w.plate.ply_of_coh, 4), ply_angle_deg=w.plate.ply_angle_deg,
                    fixed=g["fixed"], surf=g["surf"], dims=w.plate.dims,
                    grid=(2 * w.plate.grid[0], 2 * w.plate.grid[1], 2 * w.plate.grid[2]))
    Lx, Ly, H = fine.dims
    st = pi.seeded_state(fine, 5, amp=0.05, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.15, 4.0))
    ctx = pkg.pdn_init_refined(r, w.material, precision=pkg.PDN_FP32_FORCE, phi=w.phi, gravity=w.gravity)
    r.close()
    pkg.pdn_set_impactor(ctx, *w.impactor())
    pkg.pdn_set_state(ctx, *st)
    pkg.pdn_step(ctx, 2)
    o = oracle.model_for(dataclasses.replace(w, plate=fine))
    o.set_state(*st)
    assert o.step(2) == 0
    dg, vg, _ = pkg.pdn_get_state(ctx)
    do, vo, _ = o.state()
    scale = np.abs(do).max()
    assert np.abs(dg - do).max() <= 1e-4 * scale
    ctx.close()
