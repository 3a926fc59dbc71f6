"""pdn_internal_force_noalloc: the internal force for callers that cannot
allocate device memory (for example code running under a framework's
caching allocator or a fixed device-memory budget, which must not call
cudaMalloc/cudaFree itself).  Its working memory is a fixed device array
inside the library, so it needs no context.

The checks, all through the C ABI:
  * two calls in a row on the same inputs, each compared with the FP64
    oracle's internal force at the same displacement and history, within
    the tolerances of the internal-force parity test (1e-10 in FP64 element
    mode, 1e-4 in FP32 element mode, relative to the largest nodal force);
  * the damaged law through this call: a caller-supplied history copied from
    a context stepped into damage (float in FP32 element mode, double in
    FP64), with damage and plasticity on;
  * the shared array reused by a smaller mesh right after the largest mesh
    it accepts;
  * a mesh beyond the stated maximum is refused with a clear error.
Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import oracle
import pdn_inputs as pi

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-4}


def _csr(hexes, n_nodes):
    nodes = hexes.ravel().astype(np.int64)
    slots = np.arange(nodes.size, dtype=np.int64)
    order = np.lexsort((slots, nodes))
    col = slots[order].astype(np.int32)
    row = np.concatenate([[0], np.cumsum(np.bincount(nodes, minlength=n_nodes))]).astype(np.int32)
    return row, col


def _small_damage_workload(fp64):
    """16x24 hex8 per ply, 8 plies, no interfaces: 3,072 hexes, 3,825 nodes."""
    plate = pi.make_plate(12.5, 18.75, 2.2, 16, 24, pi.seeded_quasi_isotropic_layup(8, 0), 1, cohesive=False)
    mat = pi.material_im7_like_config(t_ply=2.2 / 8, seed=0)
    return pi.Workload("noalloc_plate12.5x18.75x2.2_16x24x8", plate, mat, fp64, True, True,
                       8.0, 5.5e-3 / 64, 3000.0, 0.01, 0.5, 40)


def _stepped_into_damage(pkg, w, precision):
    """A context stepped from a seeded damaging state: its displacement,
    velocity and committed history (element precision)."""
    Lx, Ly, H = w.plate.dims
    st = pi.seeded_state(w.plate, 7, amp=0.02, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.12, 1.5))
    ctx = pkg.pdn_init_mesh(w.plate, w.material, precision=precision, damage_on=True, plasticity_on=True)
    pkg.pdn_set_impactor(ctx, *w.impactor())
    pkg.pdn_set_state(ctx, *st)
    pkg.pdn_step(ctx, 40)
    d, v, _ = pkg.pdn_get_state(ctx)
    hist, _ = pkg.pdn_get_history(ctx)
    ctx.close()
    return d, v, hist


def _oracle_force(w, d, v, hist):
    """FP64 oracle internal force at (d, hist); hist in the library's
    [7][8][n_hex] layout, any float type."""
    o = oracle.Model(w.plate, w.material, damage_on=w.damage_on, plasticity_on=w.plasticity_on)
    o.set_history(np.asarray(hist, dtype=np.float64).transpose(2, 1, 0), np.zeros((0, 4)))
    o.set_state(d, v)
    f = o.internal_force()
    o.close()
    return f


def _noalloc(pkg, torch, w, d, hist, precision, damage_on=True, plasticity_on=True):
    dev = torch.device("cuda", 0)
    plate = w.plate
    row, col = _csr(plate.hex, plate.n_nodes)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    hist_d = None if hist is None else t(hist)
    f_d = torch.full((3, plate.n_nodes), float("nan"), dtype=torch.float64, device=dev)
    pkg.pdn_internal_force_noalloc(plate.n_nodes, plate.n_hex, t(plate.hex.astype(np.int32)),
                                   t(plate.ply_of_hex.astype(np.int8)), t(plate.X), t(d), hist_d, t(row), t(col),
                                   w.material, plate.ply_angle_deg, precision, damage_on, plasticity_on, f_d)
    torch.cuda.synchronize()
    return f_d.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_damaged_history_matches_oracle(precision):
    """Caller-supplied damaged history (double in FP64, float in FP32 element
    mode), damage and plasticity on; two calls in a row against the oracle."""
    import torch
    import paper_2301_05552_gb300 as pkg

    w = _small_damage_workload(fp64=precision == 0)
    d, v, hist = _stepped_into_damage(pkg, w, precision)
    assert hist.dtype == (np.float64 if precision == 0 else np.float32)
    assert (hist[:4] > 1.0).any(), "the history must be damaged"
    assert (hist[4:] != 0.0).any(), "the history must hold plastic strain"
    f_ref = _oracle_force(w, d, v, hist)
    for call in range(2):
        f = _noalloc(pkg, torch, w, d, hist, precision)
        assert np.isfinite(f).all(), f"call {call}"
        assert np.abs(f - f_ref).max() <= TOL[precision] * np.abs(f_ref).max(), f"call {call}"


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_smaller_mesh_after_largest_matches_oracle(precision):
    """The largest mesh the scratch accepts (8,192 hexes, elastic, initial
    history from the scratch), then a smaller damaged mesh in the same
    array: both against the oracle."""
    import torch
    import paper_2301_05552_gb300 as pkg

    big = pi.plain_fp64_plate()
    assert big.plate.n_hex == 8192
    db, vb = pi.seeded_state(big.plate, 21, amp=0.02, vamp=0.0)
    fb_ref = _oracle_force(big, db, vb, np.tile(np.array([1, 1, 1, 1, 0, 0, 0], dtype=np.float64)[:, None, None],
                                               (1, 8, big.plate.n_hex)))
    fb = _noalloc(pkg, torch, big, db, None, precision, damage_on=False, plasticity_on=False)
    assert np.abs(fb - fb_ref).max() <= TOL[precision] * np.abs(fb_ref).max()

    w = _small_damage_workload(fp64=precision == 0)
    d, v, hist = _stepped_into_damage(pkg, w, precision)
    f_ref = _oracle_force(w, d, v, hist)
    f = _noalloc(pkg, torch, w, d, hist, precision)
    assert np.abs(f - f_ref).max() <= TOL[precision] * np.abs(f_ref).max()


def test_noalloc_refuses_meshes_beyond_its_scratch():
    import torch
    import paper_2301_05552_gb300 as pkg

    w = pi.plain_fp64_plate()
    too_many = 8192 + 1
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.PdnError) as ei:
        pkg.pdn_internal_force_noalloc(w.plate.n_nodes, too_many, dummy, dummy, dummy, dummy, None, dummy, dummy,
                                       w.material, w.plate.ply_angle_deg, 1, False, False, dummy)
    assert ei.value.code == -1
    assert "static scratch" in str(ei.value)
