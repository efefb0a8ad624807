"""Voxel list, face nodes, incidence matrix and ports (oracle).

Sec. II.A: the K non-empty voxels each carry six face-centre nodes; faces
shared by two non-empty voxels share a node; M unique nodes in total;
N = 5K + M unknowns (Eq. 7).

Numbering conventions (also those of the library's C ABI):
* voxels: non-empty cells in raster order of the grid, x fastest, then y, then z;
* nodes: scanning voxels in that order and, per voxel, its faces in the order
  -x, +x, -y, +y, -z, +z, a face gets the next id the first time it is met;
* unknowns: [I^x (K), I^y (K), I^z (K), I^2D (K), I^3D (K), Phi (M)].

Incidence A (M x 5K), Eq. 7: entry (node of face f of voxel k, basis alpha of
voxel k) = outward flux of basis alpha through face f. With the bases
normalised so that Eq. 16-18 hold (f^x = x/dx^2, f^2D = (xi_x x - xi_y y)/dx^2,
f^3D = (xi_x x + xi_y y - 2 xi_z z)/dx^2 in local coordinates xi), the fluxes are

    x: -1 / +1 through -x / +x          2D: +1/2 through +-x, -1/2 through +-y
    y: -1 / +1 through -y / +y          3D: +1/2 through +-x and +-y, -1 through +-z
    z: -1 / +1 through -z / +z

Ports: a port lists the faces of its plus and minus terminals; a terminal
node has a known potential, so its continuity row and its Phi unknown leave
the system. A connected set of voxels with no terminal gets a gauge node.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

FLUX = np.array([
    [-1.0, 1.0, 0.0, 0.0, 0.0, 0.0],   # x
    [0.0, 0.0, -1.0, 1.0, 0.0, 0.0],   # y
    [0.0, 0.0, 0.0, 0.0, -1.0, 1.0],   # z
    [0.5, 0.5, -0.5, -0.5, 0.0, 0.0],  # 2D
    [0.5, 0.5, 0.5, 0.5, -1.0, -1.0],  # 3D
])


@dataclass
class Grid:
    Kx: int
    Ky: int
    Kz: int
    dx: float
    vox: np.ndarray          # [K] grid linear index of each voxel
    pos: np.ndarray          # [K, 3] (x, y, z) integer position
    node: np.ndarray         # [K, 6] node id of each face
    M: int
    A: sp.csr_matrix         # [M, 5K]
    lam: np.ndarray          # [K]
    sigma0: np.ndarray       # [K]
    port_plus: List[np.ndarray] = field(default_factory=list)   # node ids
    port_minus: List[np.ndarray] = field(default_factory=list)
    gauge: np.ndarray = None  # node ids fixed to 0 for floating islands

    @property
    def K(self):
        return self.vox.size

    @property
    def N(self):
        return 5 * self.K + self.M


def build_grid(structure) -> Grid:
    s = structure
    Kx, Ky, Kz = s.Kx, s.Ky, s.Kz
    occ = np.asarray(s.occ).ravel()
    vox = np.flatnonzero(occ)
    K = vox.size
    x = vox % Kx
    y = (vox // Kx) % Ky
    z = vox // (Kx * Ky)
    pos = np.stack([x, y, z], -1)
    # key of each face: (axis, integer coordinates of its plane cell)
    keys = np.empty((K, 6, 4), np.int64)
    for f in range(6):
        axis = f // 2
        plus = f % 2
        c = pos.copy()
        c[:, axis] += plus
        keys[:, f, 0] = axis
        keys[:, f, 1:] = c
    flat = keys.reshape(K * 6, 4)
    code = ((flat[:, 0] * (Kz + 2) + flat[:, 3]) * (Ky + 2) + flat[:, 2]) * (Kx + 2) + flat[:, 1]
    uniq, first, inv = np.unique(code, return_index=True, return_inverse=True)
    order = np.argsort(first, kind="stable")           # unique faces by first appearance
    rank = np.empty_like(order)
    rank[order] = np.arange(order.size)
    node = rank[inv].reshape(K, 6)
    M = uniq.size
    rows = np.repeat(node[:, None, :], 5, axis=1)        # [K, 5, 6]
    cols = (np.arange(5)[None, :, None] * K + np.arange(K)[:, None, None]) * np.ones((1, 1, 6), np.int64)
    vals = np.broadcast_to(FLUX[None, :, :], (K, 5, 6))
    mask = vals != 0
    A = sp.csr_matrix((vals[mask], (rows[mask], cols[mask])), shape=(M, 5 * K))
    A.sum_duplicates()
    gidx = -np.ones(Kx * Ky * Kz, np.int64)
    gidx[vox] = np.arange(K)
    g = Grid(Kx, Ky, Kz, s.dx, vox, pos, node, M, A,
             np.asarray(s.lam).ravel()[vox], np.asarray(s.sigma0).ravel()[vox])
    for p in s.ports:
        g.port_plus.append(_face_nodes(gidx, node, p.plus))
        g.port_minus.append(_face_nodes(gidx, node, p.minus))
    g.gauge = _gauge_nodes(g)
    return g


def _face_nodes(gidx, node, faces):
    faces = np.asarray(faces, np.int64)
    v = gidx[faces // 6]
    if np.any(v < 0):
        raise ValueError("port face on an empty voxel")
    return np.unique(node[v, faces % 6])


def _gauge_nodes(g: Grid):
    """One node per connected voxel island that touches no port terminal."""
    K = g.K
    # voxels sharing a node are connected
    r = np.repeat(np.arange(K), 6)
    c = g.node.ravel()
    B = sp.csr_matrix((np.ones(r.size), (r, c)), shape=(K, g.M))
    ncomp, lab = csg.connected_components(B @ B.T, directed=False)
    term = np.zeros(g.M, bool)
    for a in g.port_plus + g.port_minus:
        term[a] = True
    out = []
    for comp in range(ncomp):
        vs = np.flatnonzero(lab == comp)
        nodes = g.node[vs].ravel()
        if not term[nodes].any():
            out.append(int(g.node[vs[0], 0]))
    return np.array(out, np.int64)


def terminal_nodes(g: Grid):
    """All nodes whose potential is prescribed (port terminals and gauges)."""
    t = np.zeros(g.M, bool)
    for a in g.port_plus + g.port_minus:
        t[a] = True
    if g.gauge is not None and g.gauge.size:
        t[g.gauge] = True
    return t
