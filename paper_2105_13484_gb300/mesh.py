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
    V = vert_pos.shape[0]
    # --- edges: one per unordered vertex pair on a cell boundary, numbered in
    # order of first appearance (cell-major); the first cell seen is c1
    jj = np.arange(maxE)[None, :]
    valid = jj < n_on_cell[:, None]
    nn = np.maximum(n_on_cell, 1)[:, None]
    va = cell_verts
    vb = np.take_along_axis(cell_verts, (jj + 1) % nn, axis=1)
    ci, cj = np.nonzero(valid)                      # cell-major order
    a, b = va[ci, cj].astype(np.int64), vb[ci, cj].astype(np.int64)
    key = np.minimum(a, b) * V + np.maximum(a, b)
    uk, first, inv = np.unique(key, return_index=True, return_inverse=True)
    rank = np.empty(uk.size, dtype=np.int64)
    rank[np.argsort(first, kind="stable")] = np.arange(uk.size)
    eid = rank[inv]
    E = uk.size
    edgesOnCell = -np.ones((C, maxE), dtype=np.int64)
    edgesOnCell[ci, cj] = eid
    cellsOnEdge = -np.ones((E, 2), dtype=np.int64)
    vpair = np.zeros((E, 2), dtype=np.int64)
    is_first = np.zeros(eid.size, dtype=bool)
    is_first[first] = True
    cellsOnEdge[eid[is_first], 0] = ci[is_first]
    vpair[eid[is_first]] = np.stack([a[is_first], b[is_first]], axis=1)
    cellsOnEdge[eid[~is_first], 1] = ci[~is_first]
    assert (cellsOnEdge[:, 1] >= 0).all(), "mesh is not closed"
    # position of each edge in the edge list of its c1 and of its c2
    pos = np.zeros((E, 2), dtype=np.int64)
    pos[eid[is_first], 0] = cj[is_first]
    pos[eid[~is_first], 1] = cj[~is_first]

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

    # --- vertices: 3 cells, 3 edges each (cells in cell-major order of
    # appearance, edges in edge order)
    vv = cell_verts[ci, cj].astype(np.int64)
    order = np.argsort(vv, kind="stable")
    cnt = np.bincount(vv, minlength=V)
    assert (cnt == 3).all(), "every vertex must touch 3 cells"
    slot = np.arange(vv.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    cellsOnVertex = -np.ones((V, 3), dtype=np.int64)
    kiteAreasOnVertex = np.zeros((V, 3))
    cellsOnVertex[vv[order], slot] = ci[order]
    kiteAreasOnVertex[vv[order], slot] = kite[ci[order], cj[order]]
    areaTriangle = kiteAreasOnVertex.sum(axis=1)
    ve = verticesOnEdge.ravel()
    order = np.argsort(ve, kind="stable")
    cnt = np.bincount(ve, minlength=V)
    assert (cnt == 3).all()
    slot = np.arange(ve.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    edgesOnVertex = -np.ones((V, 3), dtype=np.int64)
    edgesOnVertex[ve[order], slot] = (np.arange(ve.size) // 2)[order]

    # --- TRiSK weights (Thuburn et al. 2009): walk each cell of e counter-
    # clockwise starting after e; the weight of the m-th edge is
    # s_i * (sum_{r=1..m} R_{i,v_r} - 1/2) * n_{e',i}, with s_{c2}=+1,
    # s_{c1}=-1, R = kite/areaCell and n_{e',i}=+1 if e' points out of i.
    maxE2 = 2 * (maxE - 1)
    edgesOnEdge = -np.ones((E, maxE2), dtype=np.int64)
    weightsOnEdge = np.zeros((E, maxE2))
    ee = np.arange(E)
    col0 = np.zeros(E, dtype=np.int64)
    for side, sgn in ((0, -1.0), (1, 1.0)):
        i = cellsOnEdge[:, side]
        n = n_on_cell[i].astype(np.int64)
        j0 = pos[:, side]
        racc = np.zeros(E)
        for mm in range(1, maxE):
            ok = mm < n
            jv = (j0 + mm) % np.maximum(n, 1)   # vertex v_m sits at the start of edge j0+m
            racc = np.where(ok, racc + kite[i, jv] / areaCell[i], racc)
            ep = edgesOnCell[i, jv]
            nsign = np.where(cellsOnEdge[np.maximum(ep, 0), 0] == i, 1.0, -1.0)
            col = col0 + mm - 1
            edgesOnEdge[ee[ok], col[ok]] = ep[ok]
            weightsOnEdge[ee[ok], col[ok]] = (sgn * (racc - 0.5) * nsign)[ok]
        col0 = col0 + n - 1
    nEdgesOnEdge = col0

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


# ----------------------------------------------------------------------------
# icosahedral geodesic sphere
# ----------------------------------------------------------------------------
def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    p = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t],
                  [0, -1, -t], [0, 1, -t], [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]],
                 dtype=F64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9],
                  [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2],
                  [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5], [2, 4, 11], [6, 2, 10],
                  [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return p / np.linalg.norm(p, axis=1, keepdims=True), f


def _orient_outward(p, f):
    a, b, c = p[f[:, 0]], p[f[:, 1]], p[f[:, 2]]
    out = np.sum(np.cross(b - a, c - a) * (a + b + c), axis=1) < 0
    f = f.copy()
    f[out] = f[out][:, [0, 2, 1]]
    return f


def _subdivide(p, f):
    """Split every triangle into four; new points on the unit sphere."""
    nP = p.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    key = np.minimum(e[:, 0], e[:, 1]) * nP + np.maximum(e[:, 0], e[:, 1])
    uk, first, inv = np.unique(key, return_index=True, return_inverse=True)
    mid = p[e[first, 0]] + p[e[first, 1]]
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    m = nP + inv.reshape(3, -1)          # midpoint ids of (01, 12, 20) per face
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    m01, m12, m20 = m[0], m[1], m[2]
    nf = np.concatenate([np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
                         np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)])
    return np.concatenate([p, mid]), nf


def _largest_component(cellsOnEdge, ocean):
    """Mask of the largest connected set of ocean cells (edges between ocean cells)."""
    C = ocean.size
    c1, c2 = cellsOnEdge[:, 0], cellsOnEdge[:, 1]
    keep = ocean[c1] & ocean[c2]
    parent = np.arange(C)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in zip(c1[keep], c2[keep]):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(i) for i in range(C)])
    roots[~ocean] = -1
    vals, counts = np.unique(roots[ocean], return_counts=True)
    return roots == vals[np.argmax(counts)]


def geodesic_sphere(level: int, *, R: float = 6.371e6, omega: float = 7.292e-5, land=None,
                    depth=4000.0) -> Mesh:
    """Voronoi (hexagon/pentagon) C-grid on the icosahedral geodesic grid.

    Cells are the 10 * 4**level + 2 points of the recursively bisected
    icosahedron; vertices are the circumcentres of its triangles.  Coriolis
    f = 2 Omega sin(latitude).  ``land`` is None or a function of the unit
    cell-centre vectors [C, 3] returning a boolean mask; only the largest
    connected ocean basin is kept.  ``depth`` is a constant or a function of
    the unit vectors.
    """
    p, f = _icosahedron()
    f = _orient_outward(p, f)
    for _ in range(level):
        p, f = _subdivide(p, f)
    C = p.shape[0]
    a, b, c = p[f[:, 0]], p[f[:, 1]], p[f[:, 2]]
    cc = np.cross(b - a, c - a)
    cc /= np.linalg.norm(cc, axis=1, keepdims=True)
    # incident triangles of each cell, counter-clockwise seen from outside
    tri = np.repeat(np.arange(f.shape[0]), 3)
    cel = f.ravel()
    order = np.argsort(cel, kind="stable")
    tri, cel = tri[order], cel[order]
    cnt = np.bincount(cel, minlength=C)
    assert set(np.unique(cnt)) <= {5, 6}
    ref = np.where(np.abs(p[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(ref, p)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(p, e1)
    d = cc[tri] - p[cel]
    ang = np.arctan2(np.sum(d * e2[cel], 1), np.sum(d * e1[cel], 1))
    order = np.lexsort((ang, cel))
    tri, cel = tri[order], cel[order]
    slot = np.arange(tri.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    cv = -np.ones((C, 6), dtype=np.int64)
    cv[cel, slot] = tri
    geo = _Sphere(R)
    cell_pos, vert_pos = R * p, R * cc
    full = _build(geo, cell_pos, vert_pos, cv, cnt.astype(np.int64))
    fE = 2.0 * omega * full["xEdge"][:, 2] / R
    fV = 2.0 * omega * cc[:, 2]
    ocean = np.ones(C, dtype=bool)
    if land is not None:
        ocean = ~np.asarray(land(p), dtype=bool)
        ocean = _largest_component(full["cellsOnEdge"], ocean)
    dep = depth(p) if callable(depth) else np.full(C, float(depth))
    lat = np.arcsin(np.clip(p[:, 2], -1, 1))
    lon = np.arctan2(p[:, 1], p[:, 0])
    return _cull(full, ~ocean, cell_pos, vert_pos, fE, fV, dep, "sphere",
                 f"geodesic_l{level}", extra={"latCell": lat, "lonCell": lon})
