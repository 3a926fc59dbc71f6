"""Mesh multiplication with interface elements (Sec. 2.4, Eq. mmu,
Algorithm 3): plain CPU oracle in Python (dictionaries and loops).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the benchmark's
CPU-baseline leg, never by the product package.

The paper extends Houzeaux et al.'s mesh multiplication to interface
elements and leaves the division itself to that reference.  Reading taken
here, one level of division:

* every hex8 is divided into 8: new nodes at its edge midpoints, face
  centres and centre (the isoparametric map at the midpoints of the
  reference cube: the means of 2, 4 and 8 corners), so the children are the
  parent's trilinear map restricted to the eight sub-cubes;
* every 8-node interface element is divided into 4 by planes parallel to its
  normal (Sec. 2.4): its lower and upper faces are divided exactly as the hex
  faces they coincide with, and its zero-length edges between the two faces
  are not divided (no node is created inside the interface);
* node numbering: the old nodes keep their ids; then one node per divided
  edge, in the order in which the edges first appear over (hex, local edge);
  then one per divided face, in order of first appearance over (hex, local
  face); then one per hex centre, in hex order;
* coordinates: 0.5 (Xa + Xb), 0.25 (((X0 + X1) + X2) + X3) and
  0.125 (X0 + ... + X7) summed left to right, corners in the local order of
  the hex in which the edge or face first appears;
* a new node holds the constraint bits that all its parent corners hold
  (bitwise AND), and belongs to the contact surface when all its parent
  corners do; the surface list keeps the old nodes in their order, then the
  new surface nodes in ascending id;
* hex child (ci, cj, ck) of hex e is hex 8e + ci + 2cj + 4ck (ci along the
  0-1 edge, cj along 0-3, ck along 0-4) with the parent's ply; interface
  child (ci, cj) of interface c is 4c + ci + 2cj.

These counts follow (Eq. mmu, read with n_e^0 the total element count):
n_e = 8 n_e^0 - 4 n_ELINT^0, n_n = n_n^0 + (divided edges) + (divided
faces) + (hexes).
"""
from __future__ import annotations

import numpy as np

# hex8: bottom face counter-clockwise seen from +z, then the top face
HEX_EDGES = ((0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7))
HEX_FACES = ((0, 1, 2, 3), (4, 5, 6, 7), (0, 1, 5, 4), (1, 2, 6, 5), (2, 3, 7, 6), (3, 0, 4, 7))
# reference-cube position of each corner, in half-cells (0 or 2 per axis)
_CORNER = ((0, 0, 0), (2, 0, 0), (2, 2, 0), (0, 2, 0), (0, 0, 2), (2, 0, 2), (2, 2, 2), (0, 2, 2))


def _mid(corners):
    n = len(corners)
    return tuple(sum(_CORNER[a][i] for a in corners) // n for i in range(3))


def divide_once(X, hexes, cohs, ply, fixed, surf):
    """One level.  X [3, n] float64; hexes [nh, 8], cohs [nc, 8] int;
    ply [nh]; fixed [n] uint8; surf [ns] int.  Returns the same six arrays of
    the divided mesh and (divided edges, divided faces)."""
    X = np.asarray(X, dtype=np.float64)
    n0 = X.shape[1]
    hexes = [tuple(int(v) for v in h) for h in np.asarray(hexes).reshape(-1, 8)]
    cohs = [tuple(int(v) for v in c) for c in np.asarray(cohs).reshape(-1, 8)]
    fixed = np.zeros(n0, np.uint8) if fixed is None else np.asarray(fixed, np.uint8)
    on_surf = np.zeros(n0, bool)
    on_surf[np.asarray(surf, dtype=np.int64)] = True

    # divided edges and faces in order of first appearance
    edge_id, edge_src = {}, []
    for h in hexes:
        for a, b in HEX_EDGES:
            key = (min(h[a], h[b]), max(h[a], h[b]))
            if key not in edge_id:
                edge_id[key] = n0 + len(edge_src)
                edge_src.append((h[a], h[b]))
    ne = len(edge_src)
    face_id, face_src = {}, []
    for h in hexes:
        for f in HEX_FACES:
            nodes = tuple(h[a] for a in f)
            key = tuple(sorted(nodes))
            if key not in face_id:
                face_id[key] = n0 + ne + len(face_src)
                face_src.append(nodes)
    nf = len(face_src)
    nh = len(hexes)
    n1 = n0 + ne + nf + nh

    Xn = np.zeros((3, n1))
    Xn[:, :n0] = X
    fx = np.zeros(n1, np.uint8)
    fx[:n0] = fixed
    sf = np.zeros(n1, bool)
    sf[:n0] = on_surf
    for k, (a, b) in enumerate(edge_src):
        j = n0 + k
        for i in range(3):
            Xn[i, j] = 0.5 * (X[i, a] + X[i, b])
        fx[j] = fixed[a] & fixed[b]
        sf[j] = on_surf[a] and on_surf[b]
    for k, nodes in enumerate(face_src):
        j = n0 + ne + k
        for i in range(3):
            s = X[i, nodes[0]]
            for v in nodes[1:]:
                s = s + X[i, v]
            Xn[i, j] = 0.25 * s
        bits = 7
        for v in nodes:
            bits &= int(fixed[v])
        fx[j] = bits
        sf[j] = all(on_surf[v] for v in nodes)
    for e, h in enumerate(hexes):
        j = n0 + ne + nf + e
        for i in range(3):
            s = X[i, h[0]]
            for v in h[1:]:
                s = s + X[i, v]
            Xn[i, j] = 0.125 * s
        bits = 7
        for v in h:
            bits &= int(fixed[v])
        fx[j] = bits
        sf[j] = all(on_surf[v] for v in h)

    # children of the hexes: the 3x3x3 lattice of each parent
    new_hex = np.zeros((8 * nh, 8), np.int32)
    new_ply = np.zeros(8 * nh, np.int8)
    for e, h in enumerate(hexes):
        lat = {}
        for a in range(8):
            lat[_CORNER[a]] = h[a]
        for a, b in HEX_EDGES:
            lat[_mid((a, b))] = edge_id[(min(h[a], h[b]), max(h[a], h[b]))]
        for f in HEX_FACES:
            lat[_mid(f)] = face_id[tuple(sorted(h[a] for a in f))]
        lat[(1, 1, 1)] = n0 + ne + nf + e
        for ck in range(2):
            for cj in range(2):
                for ci in range(2):
                    c = 8 * e + ci + 2 * cj + 4 * ck
                    for a in range(8):
                        p = _CORNER[a]
                        new_hex[c, a] = lat[(ci + p[0] // 2, cj + p[1] // 2, ck + p[2] // 2)]
                    new_ply[c] = ply[e]

    # children of the interface elements: 3x3 lattices of both faces
    quad = ((0, 0), (2, 0), (2, 2), (0, 2))
    new_coh = np.zeros((4 * len(cohs), 8), np.int32)
    for c, q in enumerate(cohs):
        lats = []
        for side in (q[:4], q[4:]):
            lat = {}
            for a in range(4):
                lat[quad[a]] = side[a]
            for a in range(4):
                b = (a + 1) % 4
                key = (min(side[a], side[b]), max(side[a], side[b]))
                if key not in edge_id:
                    raise ValueError(f"interface {c}: face edge {key} is not a hex edge")
                lat[((quad[a][0] + quad[b][0]) // 2, (quad[a][1] + quad[b][1]) // 2)] = edge_id[key]
            key = tuple(sorted(side))
            if key not in face_id:
                raise ValueError(f"interface {c}: face {key} is not a hex face")
            lat[(1, 1)] = face_id[key]
            lats.append(lat)
        for cj in range(2):
            for ci in range(2):
                k = 4 * c + ci + 2 * cj
                for s, lat in enumerate(lats):
                    for a in range(4):
                        new_coh[k, 4 * s + a] = lat[(ci + quad[a][0] // 2, cj + quad[a][1] // 2)]

    new_surf = np.concatenate([np.asarray(surf, dtype=np.int32),
                               np.nonzero(sf[n0:])[0].astype(np.int32) + n0])
    return Xn, new_hex, new_coh, new_ply, fx, new_surf, (ne, nf)


def multiply(X, hexes, cohs, ply, fixed, surf, ndivi: int):
    """ndivi levels of division (Algorithm 3); returns X, hex, coh, ply,
    fixed, surf of the final mesh."""
    for _ in range(ndivi):
        X, hexes, cohs, ply, fixed, surf, _ = divide_once(X, hexes, cohs, ply, fixed, surf)
    return X, np.asarray(hexes, np.int32), np.asarray(cohs, np.int32), np.asarray(ply, np.int8), \
        np.asarray(fixed, np.uint8), np.asarray(surf, np.int32)


def multiply_plate(plate, ndivi: int):
    """The same on a pdn_inputs.Plate-like object; returns a dict of arrays
    (with ply_of_coh: interface children 4c .. 4c+3 keep the parent's)."""
    X, h, c, p, f, s = multiply(plate.X, plate.hex, plate.coh, plate.ply_of_hex, plate.fixed, plate.surf, ndivi)
    pc = np.repeat(np.asarray(plate.ply_of_coh, np.int8), 4 ** ndivi)
    return dict(X=X, hex=h, coh=c, ply_of_hex=p, ply_of_coh=pc, fixed=f, surf=s)
