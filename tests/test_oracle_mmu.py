"""Pins of the mesh-multiplication oracle (oracle/mesh_multiply.py; Sec. 2.4,
Eq. mmu, Algorithm 3) against facts that do not come from it:

* one and two levels on a structured plate give the plate that the input
  generator builds directly at 2x and 4x resolution (geometry, element
  orientation, plies, constraints, contact surface, interfaces);
* children of a distorted hex fill it exactly (volumes sum to the parent's);
* the counts of Eq. mmu (elements, nodes, boundary faces) on a distorted
  plate with interfaces, edges, faces and boundary faces counted by brute
  force;
* the oracle's own impact run on the refined plate equals the run on the
  directly built fine plate (different numbering, same mesh).
"""
import numpy as np
import pytest

import oracle
import oracle.mesh_multiply as mm
import pdn_inputs as pi


def _r(x):
    return tuple(np.round(np.asarray(x, dtype=np.float64), 9))


def _geometry(X, hexes, cohs, ply, fixed, surf):
    nodes = sorted((_r(X[:, j]), int(fixed[j])) for j in range(X.shape[1]))
    hx = sorted((tuple(_r(X[:, v]) for v in h), int(p)) for h, p in zip(hexes, ply))
    ch = sorted(tuple(_r(X[:, v]) for v in c) for c in cohs)
    sf = sorted(_r(X[:, j]) for j in surf)
    return nodes, hx, ch, sf


def _plate(n, epp):
    return pi.make_plate(4.0, 6.0, 2.0, 2 * n, 3 * n, [0.0, 90.0, 90.0, 45.0], epp, cohesive=True)


@pytest.mark.parametrize("levels", [1, 2])
def test_structured_plate_equals_direct_fine_plate(levels):
    coarse = _plate(1, 1)
    fine = _plate(2 ** levels, 2 ** levels)
    got = mm.multiply_plate(coarse, levels)
    assert got["hex"].shape == fine.hex.shape and got["coh"].shape == fine.coh.shape
    assert got["X"].shape == fine.X.shape and got["surf"].shape == fine.surf.shape
    a = _geometry(got["X"], got["hex"], got["coh"], got["ply_of_hex"], got["fixed"], got["surf"])
    b = _geometry(fine.X, fine.hex, fine.coh, fine.ply_of_hex, fine.fixed, fine.surf)
    for x, y in zip(a, b):
        assert x == y
    # interfaces join two different node layers: the lower face is a face of
    # one hex, the upper face of another, with disjoint node sets
    faces = {}
    for e, h in enumerate(got["hex"]):
        for f in mm.HEX_FACES:
            faces.setdefault(tuple(sorted(int(h[k]) for k in f)), []).append(e)
    for c in got["coh"]:
        lo, hi = tuple(sorted(c[:4])), tuple(sorted(c[4:]))
        assert len(faces[lo]) == 1 and len(faces[hi]) == 1
        assert not set(lo) & set(hi)
        assert np.array_equal(got["X"][:, c[:4]], got["X"][:, c[4:]])


def _hex_volume(X, h):
    return oracle.hex8_volume(X[:, h].T)


def test_children_of_a_distorted_hex_fill_it():
    rng = np.random.default_rng(4)
    X = np.array(mm._CORNER, dtype=np.float64).T * 0.5 + rng.uniform(-0.2, 0.2, size=(3, 8))
    hexes = np.arange(8, dtype=np.int32)[None, :]
    V = _hex_volume(X, hexes[0])
    for levels in (1, 2):
        Xn, hn, cn, pn, fn, sn = mm.multiply(X, hexes, np.zeros((0, 8), np.int32), [0], None, [], levels)
        vols = np.array([_hex_volume(Xn, h) for h in hn])
        assert len(hn) == 8 ** levels and (vols > 0).all()
        assert vols.sum() == pytest.approx(V, rel=1e-12)
        # conforming: (2^levels + 1)^3 distinct nodes, none duplicated
        k = 2 ** levels + 1
        assert Xn.shape[1] == k ** 3
        assert len({_r(Xn[:, j]) for j in range(Xn.shape[1])}) == k ** 3


def _edges_faces(hexes):
    E = {tuple(sorted((h[a], h[b]))) for h in hexes for a, b in mm.HEX_EDGES}
    F = {tuple(sorted(h[a] for a in f)) for h in hexes for f in mm.HEX_FACES}
    return E, F


def _boundary_faces(hexes, cohs):
    """Hex faces not shared with another hex nor glued to an interface, and
    the zero-thickness side faces of interfaces not shared with another
    interface: (hex part, interface part)."""
    cnt = {}
    for h in hexes:
        for f in mm.HEX_FACES:
            k = tuple(sorted(int(h[a]) for a in f))
            cnt[k] = cnt.get(k, 0) + 1
    for c in cohs:
        for side in (c[:4], c[4:]):
            k = tuple(sorted(int(v) for v in side))
            cnt[k] = cnt.get(k, 0) + 1
    nb_hex = sum(1 for h in hexes for f in mm.HEX_FACES if cnt[tuple(sorted(int(h[a]) for a in f))] == 1)
    side_cnt = {}
    for c in cohs:
        for a in range(4):
            b = (a + 1) % 4
            k = tuple(sorted((int(c[a]), int(c[b]), int(c[4 + a]), int(c[4 + b]))))
            side_cnt[k] = side_cnt.get(k, 0) + 1
    nb_coh = sum(1 for v in side_cnt.values() if v == 1)
    return nb_hex, nb_coh


def test_counts_of_eq_mmu_on_a_distorted_plate_with_interfaces():
    p = pi.make_plate(3.0, 2.0, 1.5, 3, 2, [0.0, 45.0, 45.0, -45.0, 90.0], 1, cohesive=True)
    rng = np.random.default_rng(1)
    X = p.X + rng.uniform(-0.05, 0.05, size=p.X.shape) * np.array([[1.0], [1.0], [0.0]])
    # keep the coincident interface layers coincident: jitter by (x, y) position
    key = {}
    for j in range(X.shape[1]):
        k = _r(p.X[:2, j])
        key.setdefault(k, X[:2, j].copy())
        X[:2, j] = key[k]
    nh0, nc0, n0 = p.n_hex, p.n_coh, p.n_nodes
    E, F = _edges_faces([tuple(int(v) for v in h) for h in p.hex])
    nbh0, nbc0 = _boundary_faces(p.hex, p.coh)
    Xn, hn, cn, pn, fn, sn, (ne, nf) = mm.divide_once(X, p.hex, p.coh, p.ply_of_hex, p.fixed, p.surf)
    # elements: n_e = 8 n_e^0 - 4 n_ELINT^0
    assert len(hn) + len(cn) == 8 * (nh0 + nc0) - 4 * nc0
    # nodes: every hex edge and face divided once, plus one centre per hex;
    # the interfaces' own zero-length edges and side faces are never divided
    assert (ne, nf) == (len(E), len(F))
    assert Xn.shape[1] == n0 + len(E) + len(F) + nh0
    # boundary faces: n_b = 4 n_b^0 - 2 n_b,ELINT^0
    nbh1, nbc1 = _boundary_faces(hn, cn)
    assert nbh1 + nbc1 == 4 * (nbh0 + nbc0) - 2 * nbc0
    assert nbc0 > 0


def test_refined_plate_runs_like_the_direct_fine_plate():
    """The oracle's impact run (FP64, elastic with interfaces) on the once
    refined plate and on the directly built fine plate: same contact-force
    history to round-off, although nodes and elements are numbered
    differently."""
    lay = [0.0, 90.0, 90.0, 0.0]
    coarse = pi.make_plate(8.0, 8.0, 2.0, 4, 4, lay, 1, cohesive=True)
    fine = pi.make_plate(8.0, 8.0, 2.0, 8, 8, lay, 2, cohesive=True)
    got = mm.multiply_plate(coarse, 1)
    ref = pi.Plate(X=got["X"], hex=got["hex"], coh=got["coh"], ply_of_hex=got["ply_of_hex"],
                   ply_of_coh=got["ply_of_coh"], ply_angle_deg=coarse.ply_angle_deg, fixed=got["fixed"], surf=got["surf"],
                   dims=coarse.dims, grid=fine.grid)
    mat = pi.material_im7_like_config(t_ply=0.5, spread=0.0)
    runs = []
    for plate in (ref, fine):
        M = oracle.Model(plate, mat, damage_on=False)
        M.set_impactor(2.0, 2e-4, (4.0, 4.0, 2.0 + 2.0 + 0.001), (0.0, 0.0, -2000.0))
        assert M.step(300) == 0
        runs.append((M.force_history(), M.info()["dt"]))
    (fa, dta), (fb, dtb) = runs
    assert dta == pytest.approx(dtb, rel=1e-12)
    assert fb.max() > 0.0
    assert np.abs(fa - fb).max() <= 1e-9 * fb.max()
