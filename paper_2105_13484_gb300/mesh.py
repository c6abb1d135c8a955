"""Seeded synthetic meshes for the TRiSK C-grid (input generation only).

This module builds the mesh a user hands to ``sse_mesh_create``: connectivity,
geometry and the TRiSK tangential-reconstruction weights, the same data an
MPAS mesh file carries.  It contains none of the time-stepping arithmetic.
Both the CUDA path and the CPU oracle consume the arrays it returns.

Conventions (0-based int32 indices, -1 = absent):

* ``cellsOnEdge[e] = (c1, c2)``; the edge normal n_e points from c1 to c2.
* ``verticesOnEdge[e] = (v1, v2)``; the edge tangent t_e = k x n_e points from
  v1 to v2.
* ``dcEdge`` = distance between the two cell centres (dual-edge length d_e),
  ``dvEdge`` = distance between the two vertices (primal-edge length l_e).
* ``kiteAreasOnVertex[v][j]`` is the area of the kite shared by vertex v and
  ``cellsOnVertex[v][j]`` (0 where that cell is land).
* ``edgesOnEdge[e][:nEdgesOnEdge[e]]`` with ``weightsOnEdge`` define the
  tangential velocity reconstruction
  u^t_e = (1/d_e) * sum_j weightsOnEdge[e][j] * l_{e'} * u_{e'}
  (Thuburn et al. 2009, the TRiSK scheme the paper uses in Sec. 5).

Land cells are removed after the geometry is built: edges touching land carry
no flux (u = 0), so removing them from every list is the same as keeping them
with zero velocity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

I32 = np.int32
F64 = np.float64


@dataclass
class Mesh:
    nCells: int
    nEdges: int
    nVertices: int
    maxEdges: int
    maxEdges2: int
    cellsOnEdge: np.ndarray
    verticesOnEdge: np.ndarray
    nEdgesOnCell: np.ndarray
    edgesOnCell: np.ndarray
    cellsOnVertex: np.ndarray
    edgesOnVertex: np.ndarray
    nEdgesOnEdge: np.ndarray
    edgesOnEdge: np.ndarray
    weightsOnEdge: np.ndarray
    dcEdge: np.ndarray
    dvEdge: np.ndarray
    areaCell: np.ndarray
    areaTriangle: np.ndarray
    kiteAreasOnVertex: np.ndarray
    fEdge: np.ndarray
    fVertex: np.ndarray
    bottomDepth: np.ndarray
    xCell: np.ndarray = field(default=None)      # [C, 2] planar (x, y) or [C, 3] sphere
    xEdge: np.ndarray = field(default=None)
    xVertex: np.ndarray = field(default=None)
    normalEdge: np.ndarray = field(default=None)  # unit normal n_e (2-D or 3-D)
    latCell: np.ndarray = field(default=None)
    lonCell: np.ndarray = field(default=None)
    kind: str = "planar"
    name: str = ""

    def arrays(self) -> dict:
        return {k: v for k, v in self.__dict__.items() if isinstance(v, np.ndarray)}


# ----------------------------------------------------------------------------
# geometry back-ends
# ----------------------------------------------------------------------------
class _Planar:
    """Doubly periodic plane of size (Lx, Ly); vectors by minimum image."""

    def __init__(self, Lx: float, Ly: float):
        self.L = np.array([Lx, Ly])

    def rel(self, a, b):
        d = b - a
        return d - self.L * np.round(d / self.L)

    def dist(self, a, b):
        return np.linalg.norm(self.rel(a, b), axis=-1)

    def tri_area(self, a, b, c):
        """Unsigned area of triangle (a, b, c)."""
        u = self.rel(a, b)
        w = self.rel(a, c)
        return 0.5 * np.abs(u[..., 0] * w[..., 1] - u[..., 1] * w[..., 0])

    def midpoint(self, a, b):
        return a + 0.5 * self.rel(a, b)

    def normal(self, a, b, at):
        d = self.rel(a, b)
        return d / np.linalg.norm(d, axis=-1, keepdims=True)

    def tangent(self, n, at):
        return np.stack([-n[..., 1], n[..., 0]], axis=-1)


class _Sphere:
    """Sphere of radius R; points stored as 3-D vectors of length R."""

    def __init__(self, R: float):
        self.R = R

    def _u(self, a):
        return a / np.linalg.norm(a, axis=-1, keepdims=True)

    def rel(self, a, b):
        return b - a

    def dist(self, a, b):
        ua, ub = self._u(a), self._u(b)
        c = np.cross(ua, ub)
        return self.R * np.arctan2(np.linalg.norm(c, axis=-1), np.sum(ua * ub, axis=-1))

    def tri_area(self, a, b, c):
        """Spherical excess formula (Van Oosterom & Strackee) times R^2."""
        ua, ub, uc = self._u(a), self._u(b), self._u(c)
        num = np.abs(np.sum(ua * np.cross(ub, uc), axis=-1))
        den = 1.0 + np.sum(ua * ub, axis=-1) + np.sum(ub * uc, axis=-1) + np.sum(uc * ua, axis=-1)
        return 2.0 * np.arctan2(num, den) * self.R ** 2

    def midpoint(self, a, b):
        return self.R * self._u(self._u(a) + self._u(b))

    def normal(self, a, b, at):
        """Unit tangent-plane vector at `at` pointing along the great circle a->b."""
        ua, ub, ux = self._u(a), self._u(b), self._u(at)
        axis = np.cross(ua, ub)
        n = np.cross(axis, ux)
        return n / np.linalg.norm(n, axis=-1, keepdims=True)

    def tangent(self, n, at):
        k = self._u(at)
        return np.cross(k, n)


# ----------------------------------------------------------------------------
# generic Voronoi/TRiSK builder
# ----------------------------------------------------------------------------
def _build(geo, cell_pos, vert_pos, cell_verts, n_on_cell):
    """Edges, geometry, kites and TRiSK weights from CCW cell->vertex lists.

    ``cell_verts[i][j]`` lists the vertices of cell i counter-clockwise (seen
    from above / outside).  Edge j of cell i joins vertex j and vertex j+1.
    """
    C = cell_pos.shape[0]
    maxE = cell_verts.shape[1]
    # --- edges: one per unordered vertex pair on a cell boundary
    pairs = {}
    edge_cells = []
    edge_verts = []
    edgesOnCell = -np.ones((C, maxE), dtype=np.int64)
    for i in range(C):
        n = n_on_cell[i]
        for j in range(n):
            a, b = cell_verts[i, j], cell_verts[i, (j + 1) % n]
            key = (a, b) if a < b else (b, a)
            e = pairs.get(key)
            if e is None:
                e = len(edge_cells)
                pairs[key] = e
                edge_cells.append([i, -1])
                edge_verts.append([a, b])
            else:
                edge_cells[e][1] = i
            edgesOnCell[i, j] = e
    cellsOnEdge = np.array(edge_cells, dtype=np.int64)
    vpair = np.array(edge_verts, dtype=np.int64)
    E = cellsOnEdge.shape[0]
    assert (cellsOnEdge[:, 1] >= 0).all(), "mesh is not closed"
    V = vert_pos.shape[0]

    xc1 = cell_pos[cellsOnEdge[:, 0]]
    xc2 = cell_pos[cellsOnEdge[:, 1]]
    xEdge = geo.midpoint(xc1, xc2)
    dcEdge = geo.dist(xc1, xc2)
    n_e = geo.normal(xc1, xc2, xEdge)
    t_e = geo.tangent(n_e, xEdge)
    # orient vertices so that v2 lies in +t direction
    dva = geo.rel(xEdge, vert_pos[vpair[:, 0]])
    swap = np.sum(dva * t_e, axis=-1) > 0.0
    verticesOnEdge = vpair.copy()
    verticesOnEdge[swap] = vpair[swap][:, ::-1]
    dvEdge = geo.dist(vert_pos[verticesOnEdge[:, 0]], vert_pos[verticesOnEdge[:, 1]])

    # --- kites: (cell centre, edge point before v, v, edge point after v)
    kite = np.zeros((C, maxE))
    for j in range(maxE):
        valid = n_on_cell > j
        idx = np.nonzero(valid)[0]
        nn = n_on_cell[idx]
        v = cell_verts[idx, j]
        e_after = edgesOnCell[idx, j]
        e_before = edgesOnCell[idx, (j - 1) % nn]
        xc = cell_pos[idx]
        xv = vert_pos[v]
        ma = xEdge[e_after]
        mb = xEdge[e_before]
        kite[idx, j] = geo.tri_area(xc, mb, xv) + geo.tri_area(xc, xv, ma)
    areaCell = kite.sum(axis=1)

    # --- vertices: 3 cells, 3 edges each
    cellsOnVertex = -np.ones((V, 3), dtype=np.int64)
    kiteAreasOnVertex = np.zeros((V, 3))
    cnt = np.zeros(V, dtype=np.int64)
    for i in range(C):
        for j in range(n_on_cell[i]):
            v = cell_verts[i, j]
            cellsOnVertex[v, cnt[v]] = i
            kiteAreasOnVertex[v, cnt[v]] = kite[i, j]
            cnt[v] += 1
    assert (cnt == 3).all(), "every vertex must touch 3 cells"
    areaTriangle = kiteAreasOnVertex.sum(axis=1)
    edgesOnVertex = -np.ones((V, 3), dtype=np.int64)
    cnt[:] = 0
    for e in range(E):
        for v in verticesOnEdge[e]:
            edgesOnVertex[v, cnt[v]] = e
            cnt[v] += 1
    assert (cnt == 3).all()

    # --- TRiSK weights (Thuburn et al. 2009): walk each cell of e counter-
    # clockwise starting after e; the weight of the m-th edge is
    # s_i * (sum_{r=1..m} R_{i,v_r} - 1/2) * n_{e',i}, with s_{c2}=+1,
    # s_{c1}=-1, R = kite/areaCell and n_{e',i}=+1 if e' points out of i.
    maxE2 = 2 * (maxE - 1)
    edgesOnEdge = -np.ones((E, maxE2), dtype=np.int64)
    weightsOnEdge = np.zeros((E, maxE2))
    nEdgesOnEdge = np.zeros(E, dtype=np.int64)
    pos = {}
    for i in range(C):
        for j in range(n_on_cell[i]):
            pos[(i, edgesOnCell[i, j])] = j
    for e in range(E):
        c1, c2 = cellsOnEdge[e]
        cnt_e = 0
        for i, s in ((c1, -1.0), (c2, 1.0)):
            n = n_on_cell[i]
            j0 = pos[(i, e)]
            racc = 0.0
            for m in range(1, n):
                jv = (j0 + m) % n          # vertex v_m sits at the start of edge j0+m
                racc += kite[i, jv] / areaCell[i]
                ep = edgesOnCell[i, (j0 + m) % n]
                nsign = 1.0 if cellsOnEdge[ep, 0] == i else -1.0
                edgesOnEdge[e, cnt_e] = ep
                weightsOnEdge[e, cnt_e] = s * (racc - 0.5) * nsign
                cnt_e += 1
        nEdgesOnEdge[e] = cnt_e

    return dict(
        cellsOnEdge=cellsOnEdge, verticesOnEdge=verticesOnEdge, edgesOnCell=edgesOnCell,
        nEdgesOnCell=n_on_cell.astype(np.int64), cellsOnVertex=cellsOnVertex,
        edgesOnVertex=edgesOnVertex, kiteAreasOnVertex=kiteAreasOnVertex,
        areaCell=areaCell, areaTriangle=areaTriangle, dcEdge=dcEdge, dvEdge=dvEdge,
        edgesOnEdge=edgesOnEdge, weightsOnEdge=weightsOnEdge, nEdgesOnEdge=nEdgesOnEdge,
        xEdge=xEdge, normalEdge=n_e, maxE=maxE, maxE2=maxE2,
    )


def _cull(full, land, cell_pos, vert_pos, fE, fV, depth, kind, name, extra=None):
    """Remove land cells, the edges touching them and unreferenced vertices."""
    C = full["areaCell"].shape[0]
    ocean = ~land
    coe = full["cellsOnEdge"]
    keep_e = ocean[coe[:, 0]] & ocean[coe[:, 1]]
    voe = full["verticesOnEdge"]
    keep_v = np.zeros(full["areaTriangle"].shape[0], dtype=bool)
    keep_v[voe[keep_e].ravel()] = True
    cmap = -np.ones(C, dtype=np.int64)
    cmap[ocean] = np.arange(ocean.sum())
    emap = -np.ones(coe.shape[0], dtype=np.int64)
    emap[keep_e] = np.arange(keep_e.sum())
    vmap = -np.ones(keep_v.shape[0], dtype=np.int64)
    vmap[keep_v] = np.arange(keep_v.sum())

    def remap(a, m):
        out = np.where(a >= 0, m[np.maximum(a, 0)], -1)
        return out

    maxE, maxE2 = full["maxE"], full["maxE2"]
    # edges on cell: compact the present ones
    eoc = remap(full["edgesOnCell"][ocean], emap)
    nC = eoc.shape[0]
    eoc_c = -np.ones((nC, maxE), dtype=np.int64)
    neoc = np.zeros(nC, dtype=np.int64)
    for i in range(nC):
        row = eoc[i][eoc[i] >= 0]
        eoc_c[i, :row.size] = row
        neoc[i] = row.size
    # edges on edge: drop removed neighbours
    eoe = remap(full["edgesOnEdge"][keep_e], emap)
    w = full["weightsOnEdge"][keep_e]
    nE = eoe.shape[0]
    eoe_c = -np.ones((nE, maxE2), dtype=np.int64)
    w_c = np.zeros((nE, maxE2))
    neoe = np.zeros(nE, dtype=np.int64)
    for e in range(nE):
        m = eoe[e] >= 0
        k = int(m.sum())
        eoe_c[e, :k] = eoe[e][m]
        w_c[e, :k] = w[e][m]
        neoe[e] = k
    cov = remap(full["cellsOnVertex"][keep_v], cmap)
    kites = np.where(cov >= 0, full["kiteAreasOnVertex"][keep_v], 0.0)
    eov = remap(full["edgesOnVertex"][keep_v], emap)

    m = Mesh(
        nCells=int(nC), nEdges=int(nE), nVertices=int(keep_v.sum()), maxEdges=int(maxE),
        maxEdges2=int(maxE2),
        cellsOnEdge=remap(coe[keep_e], cmap).astype(I32),
        verticesOnEdge=remap(voe[keep_e], vmap).astype(I32),
        nEdgesOnCell=neoc.astype(I32), edgesOnCell=eoc_c.astype(I32),
        cellsOnVertex=cov.astype(I32), edgesOnVertex=eov.astype(I32),
        nEdgesOnEdge=neoe.astype(I32), edgesOnEdge=eoe_c.astype(I32),
        weightsOnEdge=w_c.astype(F64),
        dcEdge=full["dcEdge"][keep_e].astype(F64), dvEdge=full["dvEdge"][keep_e].astype(F64),
        areaCell=full["areaCell"][ocean].astype(F64),
        areaTriangle=full["areaTriangle"][keep_v].astype(F64),
        kiteAreasOnVertex=kites.astype(F64),
        fEdge=fE[keep_e].astype(F64), fVertex=fV[keep_v].astype(F64),
        bottomDepth=depth[ocean].astype(F64),
        xCell=cell_pos[ocean], xEdge=full["xEdge"][keep_e], xVertex=vert_pos[keep_v],
        normalEdge=full["normalEdge"][keep_e], kind=kind, name=name,
    )
    if extra:
        for k, v in extra.items():
            setattr(m, k, v[ocean])
    return m


# ----------------------------------------------------------------------------
# planar hexagonal channel
# ----------------------------------------------------------------------------
def planar_hex(nx: int, ny: int, dc: float, *, land_rows: int = 2, depth=1000.0,
               f0: float = 1.2e-4, beta: float = 0.0, periodic_y: bool = False) -> Mesh:
    """Regular hexagonal C-grid of nx x ny ocean cells with spacing ``dc``.

    Periodic in x.  With ``periodic_y=False`` the mesh is built on an
    (ny + land_rows)-row doubly periodic torus and the extra rows are land,
    which gives solid walls at the south and north ends of the channel.
    Coriolis: f = f0 + beta * (y - Ly/2) (beta plane; f-plane if beta = 0).
    ``depth`` is a constant or a function depth(x, y) of the cell centres.
    """
    nyt = ny if periodic_y else ny + land_rows
    if nyt % 2:
        raise ValueError("total row count must be even for a periodic hex lattice")
    dy = dc * math.sqrt(3.0) / 2.0
    Lx, Ly = nx * dc, nyt * dy
    geo = _Planar(Lx, Ly)
    jj, ii = np.meshgrid(np.arange(nyt), np.arange(nx), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    cell_pos = np.stack([(ii + 0.5 * (jj % 2)) * dc, jj * dy], axis=1)
    C = nx * nyt

    def cid(i, j):
        return (j % nyt) * nx + (i % nx)

    # two vertices per cell: "N" (90 deg) -> 2c, "NE" (30 deg) -> 2c+1
    r = dc / math.sqrt(3.0)
    vert_pos = np.zeros((2 * C, 2))
    vert_pos[0::2] = cell_pos + [0.0, r]
    vert_pos[1::2] = cell_pos + [r * math.cos(math.pi / 6), r * math.sin(math.pi / 6)]
    odd = jj % 2
    W = cid(ii - 1, jj)
    SW = np.where(odd == 1, cid(ii, jj - 1), cid(ii - 1, jj - 1))
    SE = np.where(odd == 1, cid(ii + 1, jj - 1), cid(ii, jj - 1))
    # CCW from 330 deg: N(SE), NE(c), N(c), NE(W), N(SW), NE(SW)
    cv = np.stack([2 * SE, 2 * np.arange(C) + 1, 2 * np.arange(C), 2 * W + 1, 2 * SW, 2 * SW + 1],
                  axis=1)
    full = _build(geo, cell_pos, vert_pos, cv, np.full(C, 6))
    fE = f0 + beta * (full["xEdge"][:, 1] - 0.5 * ny * dy)
    # unwrap each vertex next to one of its edges so that y is continuous
    e0 = full["edgesOnVertex"][:, 0]
    vert_pos = full["xEdge"][e0] + geo.rel(full["xEdge"][e0], vert_pos)
    fV = f0 + beta * (vert_pos[:, 1] - 0.5 * ny * dy)
    land = np.zeros(C, dtype=bool)
    if not periodic_y:
        land[jj >= ny] = True
    dep = depth(cell_pos[:, 0], cell_pos[:, 1]) if callable(depth) else np.full(C, float(depth))
    name = f"planar_hex_{nx}x{ny}_dc{dc:g}"
    return _cull(full, land, cell_pos, vert_pos, fE, fV, dep, "planar", name)
