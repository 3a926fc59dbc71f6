"""Properties of the CUDA path that hold at any size, checked at the
benchmark plate's full size (128x192x16 hex8 with its interfaces) through
the C ABI.

Linear momentum: every element's nodal forces sum to zero (the shape-function
derivatives sum to zero; interface tractions act in equal and opposite
pairs), so a free plate with no gravity and no contact keeps sum_j m_j v_j.
FP64 element arithmetic keeps it to rounding; FP32 element forces leave a
residual of FP32 rounding per element (about 1e-7 of the element force),
which bounds the drift far below the momentum itself.

Angular momentum: without interface elements (whose mixed-mode tractions are
not parallel to the opening), central difference keeps
sum_j m_j (X_j + d_j) x v_j of the stored state, because the internal forces
of P = S F^T with S symmetric exert no torque at any Gauss point."""
import numpy as np
import pytest

import pdn_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2301_05552_gb300 as p
    p.lib()
    return p


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-11), ("fp32", 1e-6)])
def test_free_full_size_plate_keeps_its_linear_momentum(pkg, precision, rel):
    w = pi.damage_fp32_plate()
    p = pi.make_plate(*w.plate.dims, w.plate.grid[0], w.plate.grid[1], list(w.plate.ply_angle_deg), 1,
                      cohesive=True, clamp="none")
    Lx, Ly, H = p.dims
    d0, v0 = pi.seeded_state(p, 3, amp=0.02, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.05, 4.0))
    v0 = v0 + np.array([[150.0], [-90.0], [40.0]])
    prec = pkg.PDN_FP64 if precision == "fp64" else pkg.PDN_FP32_FORCE
    ctx = pkg.pdn_init_mesh(p, w.material, precision=prec)
    # the striker far above the plate: no contact
    pkg.pdn_set_impactor(ctx, 8.0, 5.5e-3, (0.5 * Lx, 0.5 * Ly, H + 1e4), (0.0, 0.0, -1.0))
    pkg.pdn_set_state(ctx, d0, v0)
    # lumped masses from the same mesh on the host: rho V / 8 per hex corner
    X = p.X
    lo, hi = X[:, p.hex[:, 0]], X[:, p.hex[:, 6]]
    vol = np.prod(hi - lo, axis=0)
    m = np.zeros(p.n_nodes)
    np.add.at(m, p.hex.ravel(), np.repeat(w.material["rho"] * vol / 8.0, 8))
    p0 = (m * v0).sum(axis=1)
    scale = (m * np.abs(v0)).sum(axis=1).max()
    for _ in range(4):
        pkg.pdn_step(ctx, 25)
        _, v, _ = pkg.pdn_get_state(ctx)
        assert np.abs((m * v).sum(axis=1) - p0).max() <= rel * scale
    assert pkg.pdn_get_info(ctx)["step"] == 100
    ctx.close()


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_free_spinning_full_size_plate_keeps_its_angular_momentum(pkg, precision, rel):
    """The benchmark plate's mesh and layup without interface elements (plies
    bonded), free, spinning and deforming: with the stored state (d, v) of
    central difference, sum_j m_j (X_j + d_j) x v_j changes per step only by
    the internal forces' torque, zero for P = S F^T with S symmetric at every
    Gauss point; FP32 element arithmetic leaves rounding."""
    w = pi.damage_fp32_plate()
    p = pi.make_plate(*w.plate.dims, w.plate.grid[0], w.plate.grid[1], list(w.plate.ply_angle_deg), 1,
                      cohesive=False, clamp="none")
    Lx, Ly, H = p.dims
    d0, v0 = pi.seeded_state(p, 5, amp=0.02, vamp=300.0, dimple=(0.5 * Lx, 0.5 * Ly, 0.05, 4.0))
    xc = p.X.mean(axis=1, keepdims=True)
    omega = np.array([[40.0], [-30.0], [60.0]])  # rad/s: up to about 5 m/s at the corners
    v0 = v0 + np.cross(omega.T, (p.X - xc).T).T
    prec = pkg.PDN_FP64 if precision == "fp64" else pkg.PDN_FP32_FORCE
    ctx = pkg.pdn_init_mesh(p, w.material, precision=prec)
    pkg.pdn_set_impactor(ctx, 8.0, 5.5e-3, (0.5 * Lx, 0.5 * Ly, H + 1e4), (0.0, 0.0, -1.0))
    pkg.pdn_set_state(ctx, d0, v0)
    lo, hi = p.X[:, p.hex[:, 0]], p.X[:, p.hex[:, 6]]
    m = np.zeros(p.n_nodes)
    np.add.at(m, p.hex.ravel(), np.repeat(w.material["rho"] * np.prod(hi - lo, axis=0) / 8.0, 8))

    def J(d, v):
        return (m * np.cross((p.X + d).T, v.T).T).sum(axis=1)

    j0 = J(d0, v0)
    scale = (m * np.linalg.norm(p.X + d0, axis=0) * np.linalg.norm(v0, axis=0)).sum()
    for _ in range(4):
        pkg.pdn_step(ctx, 25)
        d, v, _ = pkg.pdn_get_state(ctx)
        assert np.abs(J(d, v) - j0).max() <= rel * scale
    ctx.close()


def test_contact_nodes_of_the_full_size_plate_lie_on_the_sphere(pkg):
    """The benchmark plate (FP32 elements, FP64 nodal state and contact):
    after committed steps each node of the contact set lies on the striker's
    sphere at its current centre and moves with the striker along the sphere
    normal (Dirichlet condition, Sec. 2.1; projection and state in FP64).
    The first 1,800 steps cover the start of contact (the set holds the node
    under the striker at the sampled steps); the many-node case is pinned on
    the oracle."""
    w = pi.damage_fp32_plate()
    p = w.plate
    ctx = pkg.pdn_init_mesh(p, w.material, precision=pkg.PDN_FP32_FORCE)
    R, mass, centre, vel = w.impactor()
    pkg.pdn_set_impactor(ctx, R, mass, centre, vel)
    most = 0
    for _ in range(6):
        pkg.pdn_step(ctx, 300)
        act, _ = pkg.pdn_get_contact(ctx)
        on = act.astype(bool)
        if not on.any():
            continue
        most = max(most, int(on.sum()))
        d, v, imp = pkg.pdn_get_state(ctx)
        c, wv = np.asarray(imp["centre"]), np.asarray(imp["velocity"])
        s = p.surf[on]
        x = p.X[:, s] + d[:, s]
        r = np.linalg.norm(x - c[:, None], axis=0)
        n = (x - c[:, None]) / r
        assert np.abs(r - R).max() <= 1e-12 * R
        assert np.abs(((v[:, s] - wv[:, None]) * n).sum(axis=0)).max() <= 1e-12 * np.abs(wv).max()
    assert most >= 1
    ctx.close()
