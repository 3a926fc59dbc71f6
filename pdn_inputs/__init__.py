"""Seeded synthetic inputs for the explicit impact step: structured laminated plates,
layups, material parameter sets and striker set-ups.

This module is shared by the CUDA path's binding, the oracle's tests and the
benchmark.  It holds input preparation only (node coordinates, connectivity,
ply angles, clamped-node masks, contact-surface lists, parameter values); it
computes nothing that the solver computes (no masses, time steps, strains,
stresses, damage or contact quantities).

Units: mm, N, tonne, s, MPa (the paper's material table uses t/mm^3 and MPa).

Plates follow the drop-weight coupon of Sec. 3.2 (ASTM D7136): a rectangular
laminate, one or more hex8 elements per ply through the thickness, and
zero-thickness 8-node interface elements inserted only between plies of
different angle (Sec. 3.2, "Cohesive elements are inserted at each interface
between different ply angles").  Interface nodes are duplicated so that an
interface element's bottom and top faces are distinct node sets.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np

# Hex8 local node order used throughout: bottom face counter-clockwise seen
# from +z, then the top face in the same order.  Natural coordinates of node a
# are HEX_NODE_SIGNS[a].
HEX_NODE_SIGNS = np.array(
    [[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.int8)


@dataclasses.dataclass
class Plate:
    """A structured laminated plate mesh (structure of arrays, user numbering)."""
    X: np.ndarray            # [3, n_nodes] float64 reference coordinates
    hex: np.ndarray          # [n_hex, 8] int32
    coh: np.ndarray          # [n_coh, 8] int32 (bottom face 4, top face 4)
    ply_of_hex: np.ndarray   # [n_hex] int8
    ply_of_coh: np.ndarray   # [n_coh] int8 (ply below the interface)
    ply_angle_deg: np.ndarray  # [n_plies] float64
    fixed: np.ndarray        # [n_nodes] uint8 constraint bits: 1 x, 2 y, 4 z (7 = clamped)
    surf: np.ndarray         # [n_surf] int32 top-face node ids
    dims: tuple              # (Lx, Ly, H)
    grid: tuple              # (nx, ny, nz_elements)

    @property
    def n_nodes(self) -> int:
        return self.X.shape[1]

    @property
    def n_hex(self) -> int:
        return self.hex.shape[0]

    @property
    def n_coh(self) -> int:
        return self.coh.shape[0]

    @property
    def n_surf(self) -> int:
        return self.surf.shape[0]


def seeded_quasi_isotropic_layup(n_plies: int, seed: int) -> List[float]:
    """A symmetric layup: a seeded permutation of equal numbers of 0, 45, -45
    and 90 degree plies for the lower half, mirrored about the mid-plane."""
    if n_plies % 2:
        raise ValueError("symmetric layup needs an even ply count")
    half = n_plies // 2
    base = [0.0, 45.0, -45.0, 90.0] * ((half + 3) // 4)
    base = base[:half]
    rng = np.random.default_rng(seed)
    lower = [base[i] for i in rng.permutation(half)]
    return lower + lower[::-1]


def make_plate(Lx: float, Ly: float, H: float, nx: int, ny: int,
               ply_angles: Sequence[float], elems_per_ply: int = 1,
               cohesive: bool = True, clamp: str = "edges",
               window: tuple = (125.0, 75.0), clamp_radius: float = 5.0) -> Plate:
    """Structured plate on [0,Lx]x[0,Ly]x[0,H].

    Elements are numbered x fastest, then y, then through the thickness
    (bottom to top); nodes likewise within each node layer, layers bottom to
    top.  A new node layer is created at every ply interface whose two plies
    differ in angle (when ``cohesive``), and an interface element joins the two
    coincident layers there.

    clamp = "frame" reads the drop-weight supports of Sec. 3.2 (ASTM D7136):
    the plate rests on a frame with a centred window of ``window`` (mm); the
    bottom nodes on the window's edge take its contact (z held), and the top
    nodes within ``clamp_radius`` of the window's four corners take the
    rubber-tipped clamps (all three components held).
    """
    ply_angles = [float(a) for a in ply_angles]
    n_plies = len(ply_angles)
    nz = n_plies * elems_per_ply
    dz = H / nz
    nxn, nyn = nx + 1, ny + 1
    per_layer = nxn * nyn

    # Node layers: z value of each layer; element sub-layer -> (bottom, top) layer ids.
    layer_z: List[float] = [0.0]
    elem_layers = []          # (bottom_layer, top_layer, ply)
    coh_layers = []           # (bottom_layer, top_layer, ply_below)
    cur = 0
    for p in range(n_plies):
        if p > 0 and cohesive and ply_angles[p] != ply_angles[p - 1]:
            layer_z.append(layer_z[cur])
            coh_layers.append((cur, len(layer_z) - 1, p - 1))
            cur = len(layer_z) - 1
        for s in range(elems_per_ply):
            layer_z.append((p * elems_per_ply + s + 1) * dz)
            top = len(layer_z) - 1
            elem_layers.append((cur, top, p))
            cur = top
    n_layers = len(layer_z)

    xs = np.linspace(0.0, Lx, nxn)
    ys = np.linspace(0.0, Ly, nyn)
    gx, gy = np.meshgrid(xs, ys, indexing="xy")      # [nyn, nxn]
    X = np.empty((3, n_layers * per_layer), dtype=np.float64)
    for L, z in enumerate(layer_z):
        sl = slice(L * per_layer, (L + 1) * per_layer)
        X[0, sl] = gx.ravel()
        X[1, sl] = gy.ravel()
        X[2, sl] = z

    i = np.arange(nx)
    j = np.arange(ny)
    jj, ii = np.meshgrid(j, i, indexing="ij")        # [ny, nx]
    n00 = (jj * nxn + ii).ravel()
    quad = np.stack([n00, n00 + 1, n00 + 1 + nxn, n00 + nxn], axis=1)  # CCW from +z

    hexes, plies = [], []
    for (b, t, p) in elem_layers:
        hexes.append(np.concatenate([quad + b * per_layer, quad + t * per_layer], axis=1))
        plies.append(np.full(nx * ny, p, dtype=np.int8))
    hex_conn = np.concatenate(hexes).astype(np.int32)
    ply_of_hex = np.concatenate(plies)

    cohs, cplies = [], []
    for (b, t, p) in coh_layers:
        cohs.append(np.concatenate([quad + b * per_layer, quad + t * per_layer], axis=1))
        cplies.append(np.full(nx * ny, p, dtype=np.int8))
    if cohs:
        coh_conn = np.concatenate(cohs).astype(np.int32)
        ply_of_coh = np.concatenate(cplies)
    else:
        coh_conn = np.zeros((0, 8), dtype=np.int32)
        ply_of_coh = np.zeros((0,), dtype=np.int8)

    on_edge = ((X[0] == 0.0) | (X[0] == Lx) | (X[1] == 0.0) | (X[1] == Ly))
    if clamp == "edges":
        fixed = on_edge.astype(np.uint8) * 7
    elif clamp == "bottom":
        fixed = (X[2] == 0.0).astype(np.uint8) * 7
    elif clamp == "quarter":
        # quarter-symmetry block: x = 0 and y = 0 are symmetry planes, bottom clamped
        fixed = ((X[0] == 0.0) * 1 | (X[1] == 0.0) * 2).astype(np.uint8)
        fixed[X[2] == 0.0] = 7
    elif clamp == "none":
        fixed = np.zeros(X.shape[1], dtype=np.uint8)
    elif clamp == "frame":
        fixed = np.zeros(X.shape[1], dtype=np.uint8)
        wx, wy = window
        x0, x1 = 0.5 * (Lx - wx), 0.5 * (Lx + wx)
        y0, y1 = 0.5 * (Ly - wy), 0.5 * (Ly + wy)
        hx, hy = Lx / nx, Ly / ny
        tol_x, tol_y = 0.5 * hx, 0.5 * hy
        x, y, z = X
        # nodes of the window's edge line (within half an element)
        near_x = ((np.abs(x - x0) <= tol_x) | (np.abs(x - x1) <= tol_x)) & (y >= y0 - tol_y) & (y <= y1 + tol_y)
        near_y = ((np.abs(y - y0) <= tol_y) | (np.abs(y - y1) <= tol_y)) & (x >= x0 - tol_x) & (x <= x1 + tol_x)
        fixed[(z == 0.0) & (near_x | near_y)] = 4
        top = z == layer_z[-1]
        for cx in (x0, x1):
            for cy in (y0, y1):
                fixed[top & ((x - cx) ** 2 + (y - cy) ** 2 <= clamp_radius ** 2)] = 7
    else:
        raise ValueError(clamp)
    surf = np.arange((n_layers - 1) * per_layer, n_layers * per_layer, dtype=np.int32)
    return Plate(X=X, hex=hex_conn, coh=coh_conn, ply_of_hex=ply_of_hex,
                 ply_of_coh=ply_of_coh, ply_angle_deg=np.array(ply_angles, dtype=np.float64),
                 fixed=fixed, surf=surf, dims=(Lx, Ly, H), grid=(nx, ny, nz))


# ---------------------------------------------------------------------------
# Material parameter sets.  Keys match the solver's material record.

def material_im7_like_config(t_ply: float, strengths=(2300.0, 60.0, 90.0),
                             GIc: float = 0.3, GIIc: float = 1.0,
                             spread: float = 0.05, seed: int = 0) -> Dict[str, float]:
    """The plate material of the synthetic impact workloads: E1=140 GPa,
    E2=E3=9 GPa, G12=G13=5 GPa, nu12=nu13=0.3, rho=1600 kg/m^3; the remaining
    constants (nu23, compressive strengths, fracture toughnesses, plasticity,
    fracture angle, BK exponent) from the AS4/8552 column of the paper's
    material table (Table 1).  G23 follows transverse isotropy; the interface
    penalty stiffness is the lower bound 50 E_T / t of Sec. 2.3.2 with t the
    ply thickness; interface strengths tau_I = Y_T and tau_II = S_L as in the
    AS4/8552 column."""
    E2 = 9000.0
    nu23 = 0.45
    XT, YT, SL = strengths
    GSL = GIIc
    alpha0 = 53.0
    return dict(
        rho=1.6e-9, E1=1.4e5, E2=E2, E3=E2, nu12=0.3, nu13=0.3, nu23=nu23,
        G12=5000.0, G13=5000.0, G23=E2 / (2.0 * (1.0 + nu23)),
        XT=XT, XC=1531.0, YT=YT, YC=199.8, SL=SL, alpha0_deg=alpha0,
        GXT=81.5, GXC=106.3, GYT=GIc, GYC=GSL / np.cos(np.radians(alpha0)), GSL=GSL,
        Sp=62.0, Kp=0.1936,
        GIc=GIc, GIIc=GIIc, tauI=YT, tauII=SL, eta=1.45, KI=50.0 * E2 / t_ply,
        spread=spread, seed=seed,
    )


def material_as4_8552(t_ply: float, spread: float = 0.05, seed: int = 0) -> Dict[str, float]:
    """The AS4/8552 column of the paper's material table (Table 1): elastic
    constants, strengths (Y_T and S_L as listed), fracture toughnesses,
    plasticity, interface toughnesses (tau_I = Y_T, tau_II = S_L) and the BK
    exponent.  The interface penalty stiffness follows the 50 E_T / t rule of
    Sec. 2.3.2 with t the element-layer thickness (the table's K_coh units are
    unreadable)."""
    E2 = 7630.0
    YT, SL, GIc, GIIc = 74.2, 94.36, 0.28, 0.79
    return dict(
        rho=1.59e-9, E1=128.0e3, E2=E2, E3=E2, nu12=0.35, nu13=0.35, nu23=0.45,
        G12=4358.0, G13=4358.0, G23=2631.0,
        XT=2300.0, XC=1531.0, YT=YT, YC=199.8, SL=SL, alpha0_deg=53.0,
        GXT=81.5, GXC=106.3, GYT=GIc, GYC=1.313, GSL=GIIc,
        Sp=62.0, Kp=0.1936,
        GIc=GIc, GIIc=GIIc, tauI=YT, tauII=SL, eta=1.45, KI=50.0 * E2 / t_ply,
        spread=spread, seed=seed,
    )


def material_isotropic(E: float, nu: float, rho: float) -> Dict[str, float]:
    """An isotropic elastic solid written in the orthotropic record (used by the
    Hertz and patch checks).  Strength entries are set so large that no damage
    can start."""
    G = E / (2.0 * (1.0 + nu))
    big = 1e30
    return dict(rho=rho, E1=E, E2=E, E3=E, nu12=nu, nu13=nu, nu23=nu, G12=G, G13=G, G23=G,
                XT=big, XC=big, YT=big, YC=big, SL=big, alpha0_deg=53.0,
                GXT=1.0, GXC=1.0, GYT=1.0, GYC=1.0, GSL=1.0, Sp=big, Kp=0.0,
                GIc=1.0, GIIc=1.0, tauI=big, tauII=big, eta=1.45, KI=1e6,
                spread=0.0, seed=0)


# ---------------------------------------------------------------------------
# Workloads.

@dataclasses.dataclass
class Workload:
    name: str
    plate: Plate
    material: Dict[str, float]
    fp64: bool                 # True: element forces in FP64; False: FP32 forces
    damage_on: bool
    plasticity_on: bool
    radius: float              # mm
    mass: float                # t
    speed: float               # mm/s, along -z
    gap: float                 # mm
    dt_safety: float
    steps: int
    phi: float = 1.0
    gravity: tuple = (0.0, 0.0, 0.0)
    # steps of the impact advanced before a measured window opens, so that
    # the window lies inside the contact phase (0: the window starts at rest)
    preroll: int = 0

    def impactor(self):
        Lx, Ly, H = self.plate.dims
        centre = (0.5 * Lx, 0.5 * Ly, H + self.radius + self.gap)
        velocity = (0.0, 0.0, -self.speed)
        return self.radius, self.mass, centre, velocity


def plain_fp64_plate(nx: int = 32, ny: int = 32, steps: int = 2000) -> Workload:
    """40x40x4 mm, [0/90]2s, one element per ply, clamped edges, no damage,
    rigid sphere R=8 mm, 1 kg at 1 m/s, dt = 0.5 of the stable step."""
    lay = [0.0, 90.0, 0.0, 90.0, 90.0, 0.0, 90.0, 0.0]
    plate = make_plate(40.0, 40.0, 4.0, nx, ny, lay, 1, cohesive=False)
    mat = material_im7_like_config(t_ply=0.5, spread=0.0)
    return Workload("plate40x40x4_32x32x8_fp64_elastic", plate, mat, True, False, False,
                    8.0, 1.0e-3, 1000.0, 0.01, 0.5, steps)


def damage_fp32_plate(nx: int = 128, ny: int = 192, plies: int = 16, elems_per_ply: int = 1,
                      Lx: float = 100.0, Ly: float = 150.0, H: float = 4.4,
                      mass: float = 5.5e-3, speed: float = 3000.0, seed: int = 0,
                      steps: int = 20000, fp64: bool = False,
                      strengths=(2300.0, 60.0, 90.0), preroll: int = 2400) -> Workload:
    """100x150x4.4 mm plate, seeded quasi-isotropic 16-ply layup, intralaminar
    damage with seeded +/-5% strengths, interfaces between plies of different
    angle (GIc=0.3, GIIc=1.0 N/mm), rigid sphere R=8 mm, 5.5 kg at 3 m/s.
    The pre-roll (2,400 steps, 19.7 us) ends about half way to the peak
    contact force of the 128x192x16 plate (606 N near step 4,700), with
    the first matrix damage under the striker."""
    lay = seeded_quasi_isotropic_layup(plies, seed)
    plate = make_plate(Lx, Ly, H, nx, ny, lay, elems_per_ply, cohesive=True)
    mat = material_im7_like_config(t_ply=H / plies, strengths=strengths, seed=seed)
    name = f"plate{Lx:g}x{Ly:g}x{H:g}_{nx}x{ny}x{plies * elems_per_ply}_{'fp64' if fp64 else 'fp32'}_damage"
    return Workload(name, plate, mat, fp64, True, True, 8.0, mass, speed, 0.01, 0.5, steps,
                    preroll=preroll)


def large_fp32_plate(steps: int = 5000) -> Workload:
    """The same plate refined to 400x600x32 hex8 (two elements per ply),
    5.5 kg striker at 4 m/s.  The pre-roll (2,700 steps, 15.7 us) ends about
    half way to the peak contact force (755 N near step 5,400), with about a
    hundred damaged hexes under the striker."""
    return damage_fp32_plate(nx=400, ny=600, plies=16, elems_per_ply=2, speed=4000.0,
                             steps=steps, preroll=2700)


def as4_frame_plate(nx: int = 207, ny: int = 138, Lx: float = 150.0, Ly: float = 100.0,
                    window=(125.0, 75.0), clamp_radius: float = 5.0, mass: float = 5.0e-3,
                    speed: float = 2780.0, steps: int = 20000, fp64: bool = False,
                    seed: int = 0) -> Workload:
    """The AS4/8552 drop-weight coupon of Sec. 3.2: 150x100 mm,
    [45_4/0_4/-45_4/90_4]_S with 0.181 mm plies (5.79 mm), one element per
    four-ply cluster (the 90_8 cluster in two) and 0.725 mm in plane as the
    paper's base mesh, interfaces between clusters of different angle, frame
    and clamp supports (make_plate clamp="frame"), striker R = 8 mm, 5 kg at
    2.78 m/s (19.3 J), gap 0.01 mm, gravity 9.81 m/s^2 on plate and striker,
    Tchamwa-Wielgosz phi = 1.033."""
    t_cluster = 4 * 0.181
    lay = [45.0, 0.0, -45.0, 90.0, 90.0, -45.0, 0.0, 45.0]
    plate = make_plate(Lx, Ly, 8 * t_cluster, nx, ny, lay, 1, cohesive=True, clamp="frame",
                       window=window, clamp_radius=clamp_radius)
    mat = material_as4_8552(t_ply=t_cluster, seed=seed)
    name = f"as4_plate{Lx:g}x{Ly:g}x{8 * t_cluster:.2f}_{nx}x{ny}x8_{'fp64' if fp64 else 'fp32'}_frame"
    return Workload(name, plate, mat, fp64, True, True, 8.0, mass, speed, 0.01, 0.5, steps,
                    phi=1.033, gravity=(0.0, 0.0, -9810.0))


def reduced_as4_frame_plate(nx: int = 40, ny: int = 28, mass: float = 2.0e-4, steps: int = 2000,
                            fp64: bool = True, seed: int = 0) -> Workload:
    """A cut-down AS4/8552 coupon for parity runs: the element size, layup,
    material, clamps and striker of as4_frame_plate on nx x ny elements
    (0.725 mm spacing), with the frame window and clamp radius scaled with the
    plate and, by default, the striker mass scaled with its area."""
    Lx, Ly = nx * 150.0 / 207.0, ny * 100.0 / 138.0
    return as4_frame_plate(nx=nx, ny=ny, Lx=Lx, Ly=Ly, window=(Lx * 125.0 / 150.0, Ly * 75.0 / 100.0),
                           clamp_radius=5.0 * Lx / 150.0, mass=mass, steps=steps, fp64=fp64, seed=seed)


def batch_plates(n: int = 64, seed: int = 0, hex_min: int = 8000, hex_max: int = 400000,
                 steps: int = 2000, fp64: bool = False) -> List[Workload]:
    """Independent impact cases for a batched launch: plate sizes log-uniform
    in [hex_min, hex_max] hex8 elements, seeded symmetric quasi-isotropic
    layups of 8 to 24 plies (one element per ply, t_ply = 0.275 mm), the
    in-plane spacing of the 100x150 mm plate (100/128 mm) at aspect 2:3,
    striker R = 8 mm with mass uniform in 1-6 kg and speed uniform in 1-5 m/s,
    damage and interfaces on.  Every plate has the same stable step (same
    spacing and ply thickness)."""
    rng = np.random.default_rng(seed)
    h, t_ply = 100.0 / 128.0, 0.275
    out = []
    for k in range(n):
        target = float(np.exp(rng.uniform(np.log(hex_min), np.log(hex_max))))
        plies = 2 * int(rng.integers(4, 13))
        inplane = max(target / plies, 256.0)
        nx = max(16, int(round(np.sqrt(inplane * 2.0 / 3.0))))
        ny = max(16, int(round(nx * 1.5)))
        mass = float(rng.uniform(1.0e-3, 6.0e-3))
        speed = float(rng.uniform(1000.0, 5000.0))
        s_k = seed * 1000 + k
        lay = seeded_quasi_isotropic_layup(plies, s_k)
        plate = make_plate(nx * h, ny * h, plies * t_ply, nx, ny, lay, 1, cohesive=True)
        mat = material_im7_like_config(t_ply=t_ply, seed=s_k)
        name = f"batch{n}_seed{seed}_plate{k}_{nx}x{ny}x{plies}"
        out.append(Workload(name, plate, mat, fp64, True, True, 8.0, mass, speed, 0.01, 0.5, steps))
    return out


def seeded_state(plate: Plate, seed: int, amp: float = 0.05, vamp: float = 200.0,
                 dimple=None, jitter: bool = True):
    """A smooth seeded displacement/velocity field (SoA [3, n_nodes], float64)
    for single-step checks from a non-trivial state: a few random Fourier modes
    that vanish on the plate edges, plus an optional downward dimple
    (centre_x, centre_y, depth, radius) under the striker.  Constrained
    degrees of freedom get zero.  Interface node pairs receive slightly
    different values (a seeded per-node jitter, unless ``jitter`` is False)
    so that interface jumps are non-zero."""
    rng = np.random.default_rng(seed)
    Lx, Ly, H = plate.dims
    x, y, z = plate.X
    d = np.zeros_like(plate.X)
    v = np.zeros_like(plate.X)
    for _ in range(4):
        kx, ky = rng.integers(1, 4, size=2)
        base = np.sin(kx * np.pi * x / Lx) * np.sin(ky * np.pi * y / Ly)
        for c in range(3):
            a, b = rng.normal(size=2)
            tilt = 1.0 + 0.3 * (z / H - 0.5) * rng.normal()
            d[c] += amp * (0.2 if c < 2 else 1.0) * a * base * tilt
            v[c] += vamp * (0.2 if c < 2 else 1.0) * b * base
    if dimple is not None:
        cx, cy, depth, rad = dimple
        r2 = ((x - cx) ** 2 + (y - cy) ** 2) / rad ** 2
        d[2] -= depth * np.exp(-r2) * (0.6 + 0.4 * z / H)
    if jitter:
        d += rng.normal(size=plate.X.shape) * amp * 1e-3
    for c in range(3):
        held = ((plate.fixed >> c) & 1).astype(bool)
        d[c, held] = 0.0
        v[c, held] = 0.0
    return d, v
