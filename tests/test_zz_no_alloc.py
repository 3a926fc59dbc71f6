"""pdn_internal_force_noalloc: the internal force for callers that cannot
allocate device memory (for example code running under a framework's
caching allocator or a fixed device-memory budget, which must not call
cudaMalloc/cudaFree itself).  Its working memory is a fixed device array
inside the library, so it needs no context.

The check: through the C ABI, two calls in a row on the same inputs, each
compared with pdn_internal_force of an ordinary context holding the same
mesh and displacement, within the tolerances of the internal-force parity
test (1e-10 in FP64 element mode, 1e-4 in FP32 element mode, relative to the
largest nodal force); and a mesh beyond the stated maximum is refused with a
clear error.  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import pdn_inputs as pi

pytestmark = pytest.mark.gpu


def _csr(hexes, n_nodes):
    nodes = hexes.ravel().astype(np.int64)
    slots = np.arange(nodes.size, dtype=np.int64)
    order = np.lexsort((slots, nodes))
    col = slots[order].astype(np.int32)
    row = np.concatenate([[0], np.cumsum(np.bincount(nodes, minlength=n_nodes))]).astype(np.int32)
    return row, col


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_noalloc_matches_context_internal_force(precision, tol):
    import torch
    import paper_2301_05552_gb300 as pkg

    w = pi.plain_fp64_plate()          # 8,192 hexes, 9,801 nodes: within the stated maximum
    plate = w.plate
    mat = w.material
    d, v = pi.seeded_state(plate, 21, amp=0.02, vamp=0.0)
    ctx = pkg.pdn_init_mesh(plate, mat, precision=precision, damage_on=False, plasticity_on=False)
    pkg.pdn_set_state(ctx, d, v)
    f_ref = pkg.pdn_internal_force(ctx)
    ctx.close()

    dev = torch.device("cuda", 0)
    row, col = _csr(plate.hex, plate.n_nodes)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    hex_d, ply_d = t(plate.hex.astype(np.int32)), t(plate.ply_of_hex.astype(np.int8))
    X_d, d_d = t(plate.X), t(d)
    row_d, col_d = t(row), t(col)
    for call in range(2):
        f_d = torch.full((3, plate.n_nodes), float("nan"), dtype=torch.float64, device=dev)
        pkg.pdn_internal_force_noalloc(plate.n_nodes, plate.n_hex, hex_d, ply_d, X_d, d_d, None, row_d, col_d,
                                       mat, plate.ply_angle_deg, precision, False, False, f_d)
        torch.cuda.synchronize()
        f = f_d.cpu().numpy()
        assert np.isfinite(f).all(), f"call {call}"
        assert np.abs(f - f_ref).max() <= tol * np.abs(f_ref).max(), f"call {call}"


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
