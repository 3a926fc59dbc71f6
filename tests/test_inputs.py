"""The synthetic AS4/8552 drop-weight coupon (Sec. 3.2, Table 1) that stands
in for the paper's experiment: geometry, layup, interfaces, supports and
striker as the paper states them.  Host logic only, no GPU."""
import numpy as np
import pytest

import pdn_inputs as pi


@pytest.fixture(scope="module")
def coupon():
    return pi.as4_frame_plate()


def test_geometry_layup_and_interfaces(coupon):
    """150 x 100 mm, [45_4/0_4/-45_4/90_4]_S of 0.181 mm plies (5.792 mm),
    one element per 4-ply cluster on a 0.725 mm grid, interfaces only
    between clusters of different angle (six of the seven cluster pairs)."""
    p = coupon.plate
    assert p.dims == pytest.approx((150.0, 100.0, 32 * 0.181), rel=1e-12)
    assert list(p.ply_angle_deg) == [45.0, 0.0, -45.0, 90.0, 90.0, -45.0, 0.0, 45.0]
    assert p.n_hex == 207 * 138 * 8
    assert p.n_coh == 6 * 207 * 138
    assert p.n_nodes == 208 * 139 * (9 + 6)
    assert 150.0 / 207 == pytest.approx(0.7246, abs=1e-4) and 100.0 / 138 == pytest.approx(0.7246, abs=1e-4)
    # interface faces coincide, and no interface sits between the two 90 clusters
    assert np.array_equal(p.X[:, p.coh[:, :4]], p.X[:, p.coh[:, 4:]])
    zc = np.unique(p.X[2, p.coh[:, 0]])
    assert len(zc) == 6 and not np.any(np.isclose(zc, 4 * 4 * 0.181))


def test_frame_window_and_clamps(coupon):
    """The plate rests on a frame with a centred 125 x 75 mm window: bottom
    nodes on the window's edge hold z only; top nodes within 5 mm of the
    window's four corners hold every component; nothing else is held."""
    p = coupon.plate
    x, y, z = p.X
    f = p.fixed
    h = 150.0 / 207
    x0, x1, y0, y1 = 12.5, 137.5, 12.5, 87.5
    held_z = f == 4
    assert held_z.any() and np.all(z[held_z] == 0.0)
    on_x = np.minimum(np.abs(x - x0), np.abs(x - x1)) <= 0.5 * h
    on_y = np.minimum(np.abs(y - y0), np.abs(y - y1)) <= 0.5 * h
    inside = (x >= x0 - 0.5 * h) & (x <= x1 + 0.5 * h) & (y >= y0 - 0.5 * h) & (y <= y1 + 0.5 * h)
    assert np.array_equal(held_z, (z == 0.0) & inside & (on_x | on_y))
    clamped = f == 7
    assert np.all(z[clamped] == p.dims[2])
    counts = []
    for cx in (x0, x1):
        for cy in (y0, y1):
            near = (x - cx) ** 2 + (y - cy) ** 2 <= 25.0
            counts.append(int((clamped & near).sum()))
            assert np.array_equal(clamped & near, near & (z == p.dims[2]))
    assert len(set(counts)) == 1 and sum(counts) == int(clamped.sum())
    assert set(np.unique(f)) == {0, 4, 7}


def test_striker_gravity_and_integrator(coupon):
    """R = 8 mm, 5 kg at 2.78 m/s (19.3 J) from 0.01 mm above the plate
    centre, gravity on plate and striker, Tchamwa-Wielgosz phi = 1.033."""
    R, mass, centre, vel = coupon.impactor()
    Lx, Ly, H = coupon.plate.dims
    assert R == 8.0 and mass == 5.0e-3
    assert centre == pytest.approx((0.5 * Lx, 0.5 * Ly, H + R + 0.01), rel=1e-12)
    assert vel == (0.0, 0.0, -2780.0)
    assert 0.5 * mass * 2780.0 ** 2 / 1000.0 == pytest.approx(19.3, abs=0.05)  # N mm -> J
    assert coupon.gravity == (0.0, 0.0, -9810.0) and coupon.phi == 1.033
    # the contact surface is the top face
    p = coupon.plate
    assert np.all(p.X[2, p.surf] == H) and p.n_surf == 208 * 139


def test_batch_of_64_plates_recipe():
    """The batched workload: 64 seeded plates whose sizes are drawn
    log-uniformly in 8k-400k hex8 and rounded to whole in-plane grids
    (7,776 to 396,396 hex8, 6.23 M in all), 8-24 plies, strikers of 1-6 kg
    at 1-5 m/s, one stable step for all (same spacing and ply thickness)."""
    ws = pi.batch_plates()
    assert len(ws) == 64
    nh = np.array([w.plate.n_hex for w in ws])
    assert nh.min() == 7776 and nh.max() == 396396 and nh.sum() == 6229848
    assert all(8 <= len(w.plate.ply_angle_deg) <= 24 for w in ws)
    assert all(1.0e-3 <= w.mass <= 6.0e-3 and 1000.0 <= w.speed <= 5000.0 for w in ws)
    h = {round(w.plate.dims[0] / w.plate.grid[0], 12) for w in ws}
    t = {round(w.plate.dims[2] / len(w.plate.ply_angle_deg), 12) for w in ws}
    assert len(h) == 1 and len(t) == 1
    assert len({w.name for w in ws}) == 64


def test_large_plate_recipe():
    """The 100x150x4.4 mm plate refined to 400x600x32 hex8 (two elements per
    ply, 7.68 M hex), interfaces between plies of different angle, 5.5 kg at
    4 m/s."""
    w = pi.large_fp32_plate()
    p = w.plate
    assert p.dims == pytest.approx((100.0, 150.0, 4.4))
    assert p.n_hex == 400 * 600 * 32
    n_if = sum(1 for a, b in zip(p.ply_angle_deg[:-1], p.ply_angle_deg[1:]) if a != b)
    assert len(p.ply_angle_deg) == 16 and p.n_coh == n_if * 400 * 600
    assert p.n_nodes == 401 * 601 * (33 + n_if)
    R, mass, centre, vel = w.impactor()
    assert (R, mass, vel) == (8.0, 5.5e-3, (0.0, 0.0, -4000.0))
