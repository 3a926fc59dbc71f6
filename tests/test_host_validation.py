"""Host-side argument checks of pdn_init_mesh and pdn_mesh_multiply
(include/pdn.h, include/pdn_mmu.h).  Every check runs before the library
touches a device, so these tests run without a GPU: each malformed input
must come back as PDN_E_ARG (-1) with a message that names the problem."""
import ctypes

import numpy as np
import pytest

import pdn_inputs as pi


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


def _plate(cohesive=True):
    return pi.make_plate(4.0, 4.0, 2.0, 2, 2, [0.0, 90.0], 1, cohesive=cohesive)


def _mat():
    return pi.material_im7_like_config(t_ply=1.0)


def _init_error(pkg, plate, mat=None, **kw):
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_init_mesh(plate, _mat() if mat is None else mat, **kw)
    assert e.value.code == -1
    return str(e.value)


def _raw_init(pkg, m):
    """pdn_init_mesh on a hand-made descriptor (sizes without arrays)."""
    L = pkg.lib()
    mat = pkg._material(_mat())
    o = pkg._options(pkg.PDN_FP32_FORCE, 1, 1, 8, 1.0, 0.0, 0.5, (0.0, 0.0, 0.0), 16, None)
    h = ctypes.c_void_p()
    rc = L.pdn_init_mesh(ctypes.byref(h), ctypes.byref(m), ctypes.byref(mat), ctypes.byref(o))
    return rc, (L.pdn_last_error(None) or b"").decode()


def test_sizes_beyond_32_bit_ids_are_refused(pkg):
    m = pkg.MeshDesc()
    m.n_nodes, m.n_hex, m.n_coh, m.n_surf = 2 ** 31, 1, 0, 0
    rc, msg = _raw_init(pkg, m)
    assert rc == -1 and "32-bit" in msg
    m.n_nodes, m.n_hex, m.n_coh = 100, 2 ** 27, 2 ** 27  # 8 (n_hex + n_coh) slots overflow
    rc, msg = _raw_init(pkg, m)
    assert rc == -1 and "32-bit" in msg


def test_empty_or_negative_counts_and_missing_arrays(pkg):
    m = pkg.MeshDesc()
    m.n_nodes, m.n_hex = 8, 0
    rc, msg = _raw_init(pkg, m)
    assert rc == -1 and "n_hex > 0" in msg
    m.n_hex, m.n_coh = 1, -1
    rc, msg = _raw_init(pkg, m)
    assert rc == -1 and "n_coh >= 0" in msg
    m.n_coh = 0
    rc, msg = _raw_init(pkg, m)  # no X, hex, plies
    assert rc == -1 and "required" in msg
    p = _plate()
    desc, keep = pkg._mesh_desc(p)
    desc.coh = None
    rc, msg = _raw_init(pkg, desc)
    assert rc == -1 and "coh is NULL" in msg
    desc, keep = pkg._mesh_desc(p)
    desc.surf = None
    rc, msg = _raw_init(pkg, desc)
    assert rc == -1 and "surf is NULL" in msg
    desc, keep = pkg._mesh_desc(p)
    desc.n_plies = 0
    rc, msg = _raw_init(pkg, desc)
    assert rc == -1 and "n_plies" in msg


def test_ids_out_of_range(pkg):
    p = _plate()
    p.hex = p.hex.copy()
    p.hex[1, 3] = -1
    assert "hex node id" in _init_error(pkg, p)
    p = _plate()
    p.coh = p.coh.copy()
    p.coh[0, 5] = p.n_nodes
    assert "interface node id" in _init_error(pkg, p)
    p = _plate()
    p.ply_of_hex = p.ply_of_hex.copy()
    p.ply_of_hex[0] = len(p.ply_angle_deg)
    assert "ply id" in _init_error(pkg, p)
    p = _plate()
    p.surf = p.surf.copy()
    p.surf[-1] = p.n_nodes
    assert "surface node id" in _init_error(pkg, p)
    p = _plate()
    p.surf = np.concatenate([p.surf, p.surf[3:4]])
    assert "duplicate" in _init_error(pkg, p)


def test_unknown_precision(pkg):
    assert "precision" in _init_error(pkg, _plate(), precision=7)


def test_interface_faces_must_coincide(pkg):
    """Zero-thickness interface elements (Sec. 2.3): an upper face that is not
    the lower face in the reference configuration is refused."""
    p = _plate()
    X = p.X.copy()
    X[2, p.coh[0, 6]] += 1e-3
    p.X = X
    assert "zero thickness" in _init_error(pkg, p)


def test_constraint_bits_and_material_signs(pkg):
    p = _plate()
    p.fixed = p.fixed.copy()
    p.fixed[0] = 8
    assert "constraint bits" in _init_error(pkg, p)
    mat = _mat()
    mat["E2"] = 0.0
    assert "moduli" in _init_error(pkg, _plate(), mat=mat)
    mat = _mat()
    mat["GIIc"] = -1.0
    assert "interface constants" in _init_error(pkg, _plate(), mat=mat)


def test_mesh_multiply_refuses_bad_meshes_before_the_device(pkg):
    """pdn_mesh_multiply (Algorithm 3): levels outside 0..6 and ids out of
    range are refused on the host."""
    p = _plate()
    for levels in (-1, 7):
        with pytest.raises(pkg.PdnError) as e:
            pkg.pdn_mesh_multiply(p, levels)
        assert e.value.code == -1 and "ndivi" in str(e.value)
    bad = _plate()
    bad.hex = bad.hex.copy()
    bad.hex[0, 0] = bad.n_nodes
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_mesh_multiply(bad, 1)
    assert e.value.code == -1 and "hex node id" in str(e.value)
    bad = _plate()
    bad.ply_of_hex = bad.ply_of_hex.copy()
    bad.ply_of_hex[2] = -1
    with pytest.raises(pkg.PdnError) as e:
        pkg.pdn_mesh_multiply(bad, 1)
    assert e.value.code == -1 and "ply index" in str(e.value)
