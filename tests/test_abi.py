"""The C-ABI library loads and exports every entry point that include/*.h
declare, and the Python binding exposes the same names.  No GPU work: only
symbol lookups and argument checks that return before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(pdn_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pdn_init_mesh", "pdn_set_impactor", "pdn_step", "pdn_contact_force", "pdn_damage_field"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2301_05552_gb300 as pkg
    L = pkg.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in pkg.EXPORTS
        assert callable(getattr(pkg, name)), name


def test_init_rejects_null_arguments_without_touching_the_device():
    import paper_2301_05552_gb300 as pkg
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.pdn_init_mesh(ctypes.byref(h), None, None, None) == -1
    assert b"required" in L.pdn_last_error(None)
    assert L.pdn_init_mesh(None, None, None, None) == -1
    assert L.pdn_step(None, 1) == -1
    assert L.pdn_get_info(None, None) == -1
    L.pdn_destroy(None)


def test_batch_init_rejects_bad_arguments_without_touching_the_device():
    import paper_2301_05552_gb300 as pkg
    L = pkg.lib()
    h = ctypes.c_void_p()
    assert L.pdn_batch_init(ctypes.byref(h), 0, None, None, None) == -1
    assert b"n_plates" in L.pdn_batch_last_error(None)
    assert L.pdn_batch_init(ctypes.byref(h), 2, None, None, None) == -1
    assert b"required" in L.pdn_batch_last_error(None)
    assert L.pdn_batch_init(None, 2, None, None, None) == -1
    assert L.pdn_batch_step(None, 1) == -1
    assert L.pdn_batch_get_info(None, None) == -1
    assert L.pdn_batch_plate(None, 0) is None
    assert L.pdn_batch_test_barrier_timeout(None, 1.0) == -1
    L.pdn_batch_destroy(None)


def test_struct_layouts_match_header_sizes():
    """ctypes mirrors of the header structs have the C sizes (all fields are
    8-byte scalars or pointers except the documented int32 members)."""
    import paper_2301_05552_gb300 as pkg
    assert ctypes.sizeof(pkg.MeshDesc) == 4 * 8 + 5 * 8 + 8 + 2 * 8
    assert ctypes.sizeof(pkg.Material) == 31 * 8
    assert ctypes.sizeof(pkg.Options) == 4 * 4 + 3 * 8 + 3 * 8 + 8 + 8
    assert ctypes.sizeof(pkg.Info) == 5 * 8 + 8 * 8 + 6 * 4 + 12 * 8
    assert ctypes.sizeof(pkg.BatchInfo) == 10 * 4 + 4 * 8 + 2 * 8 + 16 * 8 + 3 * 16 * 4 + 2 * 4 + 16 * 4
    assert ctypes.sizeof(pkg.RefinedInfo) == 6 * 8 + 2 * 4 + 8


def test_plate_generator_topology():
    import pdn_inputs as pi
    w = pi.damage_fp32_plate()
    p = w.plate
    assert p.n_hex == 128 * 192 * 16
    n_if = sum(1 for a, b in zip(p.ply_angle_deg[:-1], p.ply_angle_deg[1:]) if a != b)
    assert p.n_coh == n_if * 128 * 192
    assert p.n_nodes == 129 * 193 * (17 + n_if)
    assert p.n_surf == 129 * 193
    # interface element faces are coincident node pairs
    Xb = p.X[:, p.coh[:, :4]]
    Xt = p.X[:, p.coh[:, 4:]]
    assert np.array_equal(Xb, Xt)
    # every hex has positive volume orientation (top face above bottom)
    z = p.X[2]
    assert np.all(z[p.hex[:, 4:]] > z[p.hex[:, :4]])
    # the layup is symmetric and quasi-isotropic
    ang = list(p.ply_angle_deg)
    assert ang == ang[::-1]
    assert sorted(ang[:8]) == [-45.0, -45.0, 0.0, 0.0, 45.0, 45.0, 90.0, 90.0]
    w1 = pi.plain_fp64_plate()
    assert (w1.plate.n_hex, w1.plate.n_nodes, w1.plate.n_surf) == (8192, 9801, 1089)


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_headers_compile_as_plain_c_and_cpp(lang, std):
    """Each public header stands alone as C99 and as C++17 with strict
    warnings: the boundary is plain C types, pointers and sizes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = f'#include "{h}"\n'
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                            "-I", os.path.join(ROOT, "include"), "-"], input=src, capture_output=True, text=True)
        assert r.returncode == 0, (h, r.stderr)
