"""Seeded synthetic nested simplex meshes (inputs only; no wave arithmetic).

The method discretises the domain with a d-simplex mesh and a hierarchy of
coarser meshes nested in it by regular refinement (Sec. II-B; Sec. III
"Numerical experiments", Fig. 2).  This module builds such hierarchies:

* ``square_mesh``    - [-1,1]^2 grid of right triangles (uniform, one diagonal
                       direction), refined from a coarse grid.
* ``asteroid_mesh``  - 2D star-shaped domain r(t) = 1 + 0.1 sin 3t + 0.05 cos 5t
                       meshed by concentric rings, refined uniformly.
* ``ellipsoid_mesh`` - 3D ellipsoid, Kuhn-triangulated cube grid mapped onto a
                       ball and scaled, refined by Bey's regular 1->8 rule.

Refinement halves every edge (midpoint nodes appended after the parent's
nodes, so the N coarse nodes keep ids 0..N-1, as Sec. II-B requires of the
nested meshes) and numbers the children of parent cell p as
``2**d * p + k``.  Boundary midpoints are not projected onto the curved
boundary, so nesting stays exact and the boundary stays the level-0 polygon.

This module is shared by the oracle and the CUDA path as an input source; it
computes geometry only, nothing of the wave scheme.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class NestedMesh:
    """A nested simplex mesh hierarchy, finest level materialised.

    coords      float64 [n, d]      finest-level node coordinates
    cells       int32   [m, d+1]    finest-level cells
    bnd         int32   [nb, d]     finest-level boundary facets
    cell_parent list of int32 arrays; cell_parent[l-1][c] is the level-(l-1)
                parent of level-l cell c, for l = 1..L
    n_cells     list of int; cells per level 0..L
    n_nodes     list of int; nodes per level 0..L (coarse nodes are a prefix)
    """

    dim: int
    coords: np.ndarray
    cells: np.ndarray
    bnd: np.ndarray
    cell_parent: list
    n_cells: list
    n_nodes: list

    @property
    def n_levels(self) -> int:
        return len(self.n_cells)

    def ancestor(self, level: int) -> np.ndarray:
        """Map finest cell -> its ancestor cell on ``level`` (int64 [m])."""
        L = self.n_levels - 1
        anc = np.arange(self.n_cells[L], dtype=np.int64)
        for l in range(L, level, -1):
            anc = self.cell_parent[l - 1][anc].astype(np.int64)
        return anc

    def mean_edge_length(self) -> float:
        """Mean length over the unique edges of the finest mesh."""
        d = self.dim
        pairs = [(a, b) for a in range(d + 1) for b in range(a + 1, d + 1)]
        e = np.concatenate([self.cells[:, [a, b]] for a, b in pairs])
        e = np.sort(e, axis=1).astype(np.int64)
        key = np.unique(e[:, 0] * self.coords.shape[0] + e[:, 1])
        a, b = key // self.coords.shape[0], key % self.coords.shape[0]
        return float(np.linalg.norm(self.coords[a] - self.coords[b], axis=1).mean())


def _boundary_facets(cells: np.ndarray, dim: int) -> np.ndarray:
    """Facets that belong to exactly one cell, in a deterministic order."""
    k = dim + 1
    faces = np.concatenate(
        [np.delete(cells, j, axis=1) for j in range(k)]).astype(np.int64)
    key_sorted = np.sort(faces, axis=1)
    _, first, counts = np.unique(key_sorted, axis=0, return_index=True,
                                 return_counts=True)
    once = np.sort(first[counts == 1])
    return faces[once].astype(np.int32)


def _edge_midpoints(n: int, edges: np.ndarray):
    """Unique edges of an [E,2] list -> (ids of the midpoint node per input
    edge, endpoints a, b of each unique edge in order of new node id)."""
    es = np.sort(edges, axis=1).astype(np.int64)
    key = es[:, 0] * n + es[:, 1]
    uniq, inv = np.unique(key, return_inverse=True)
    return n + inv.reshape(-1), uniq // n, uniq % n, uniq


def _lookup_mid(n: int, uniq: np.ndarray, u: np.ndarray, v: np.ndarray):
    lo, hi = np.minimum(u, v).astype(np.int64), np.maximum(u, v).astype(np.int64)
    pos = np.searchsorted(uniq, lo * n + hi)
    assert np.all(uniq[pos] == lo * n + hi), "boundary edge missing from cells"
    return n + pos


def refine2d(coords, cells, bnd):
    """One regular 1->4 refinement of a triangle mesh (children 4p+k)."""
    n, m = coords.shape[0], cells.shape[0]
    a, b, c = cells[:, 0], cells[:, 1], cells[:, 2]
    edges = np.concatenate([np.stack([a, b], 1), np.stack([b, c], 1),
                            np.stack([c, a], 1)])
    mid, ea, eb, uniq = _edge_midpoints(n, edges)
    mab, mbc, mca = mid[:m], mid[m:2 * m], mid[2 * m:]
    new_coords = np.concatenate([coords, 0.5 * (coords[ea] + coords[eb])])
    ch = np.stack([
        np.stack([a, mab, mca], 1),
        np.stack([mab, b, mbc], 1),
        np.stack([mca, mbc, c], 1),
        np.stack([mab, mbc, mca], 1),
    ], 1).reshape(4 * m, 3).astype(np.int32)
    parent = (np.arange(4 * m) // 4).astype(np.int32)
    u, v = bnd[:, 0], bnd[:, 1]
    w = _lookup_mid(n, uniq, u, v)
    new_bnd = np.stack([np.stack([u, w], 1), np.stack([w, v], 1)],
                       1).reshape(-1, 2).astype(np.int32)
    return new_coords, ch, new_bnd, parent


def refine3d(coords, cells, bnd):
    """One regular 1->8 refinement of a tetrahedral mesh (Bey's rule: the
    inner octahedron is cut along the diagonal between the midpoints of
    edges 02 and 13; children 8p+k)."""
    n, m = coords.shape[0], cells.shape[0]
    x0, x1, x2, x3 = (cells[:, i] for i in range(4))
    pairs = [(x0, x1), (x0, x2), (x0, x3), (x1, x2), (x1, x3), (x2, x3)]
    edges = np.concatenate([np.stack(p, 1) for p in pairs])
    mid, ea, eb, uniq = _edge_midpoints(n, edges)
    m01, m02, m03, m12, m13, m23 = (mid[i * m:(i + 1) * m] for i in range(6))
    new_coords = np.concatenate([coords, 0.5 * (coords[ea] + coords[eb])])
    ch = np.stack([
        np.stack([x0, m01, m02, m03], 1),
        np.stack([m01, x1, m12, m13], 1),
        np.stack([m02, m12, x2, m23], 1),
        np.stack([m03, m13, m23, x3], 1),
        np.stack([m01, m02, m03, m13], 1),
        np.stack([m01, m02, m12, m13], 1),
        np.stack([m02, m03, m13, m23], 1),
        np.stack([m02, m12, m13, m23], 1),
    ], 1).reshape(8 * m, 4).astype(np.int32)
    parent = (np.arange(8 * m) // 8).astype(np.int32)
    u, v, w = bnd[:, 0], bnd[:, 1], bnd[:, 2]
    muv = _lookup_mid(n, uniq, u, v)
    mvw = _lookup_mid(n, uniq, v, w)
    muw = _lookup_mid(n, uniq, u, w)
    new_bnd = np.stack([
        np.stack([u, muv, muw], 1),
        np.stack([muv, v, mvw], 1),
        np.stack([muw, mvw, w], 1),
        np.stack([muv, mvw, muw], 1),
    ], 1).reshape(-1, 3).astype(np.int32)
    return new_coords, ch, new_bnd, parent


def build_hierarchy(dim, coords, cells, n_refine) -> NestedMesh:
    """Refine a level-0 mesh ``n_refine`` times and record the nesting."""
    coords = np.asarray(coords, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int32)
    bnd = _boundary_facets(cells, dim)
    parents, n_cells, n_nodes = [], [cells.shape[0]], [coords.shape[0]]
    ref = refine2d if dim == 2 else refine3d
    for _ in range(n_refine):
        coords, cells, bnd, parent = ref(coords, cells, bnd)
        parents.append(parent)
        n_cells.append(cells.shape[0])
        n_nodes.append(coords.shape[0])
    return NestedMesh(dim, coords, cells, bnd, parents, n_cells, n_nodes)


# ---------------------------------------------------------------- 2D square
def rectangle_level0(nx: int, ny: int, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0):
    """[x0,x1]x[y0,y1] grid of nx*ny rectangles, each cut by its
    lower-left/upper-right diagonal into two right triangles (CCW)."""
    tx = np.linspace(x0, x1, nx + 1)
    ty = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(tx, ty, indexing="xy")
    coords = np.stack([X.ravel(), Y.ravel()], 1)
    idx = np.arange((nx + 1) * (ny + 1)).reshape(ny + 1, nx + 1)
    v00, v10 = idx[:-1, :-1].ravel(), idx[:-1, 1:].ravel()
    v01, v11 = idx[1:, :-1].ravel(), idx[1:, 1:].ravel()
    tri = np.stack([np.stack([v00, v10, v11], 1),
                    np.stack([v00, v11, v01], 1)], 1).reshape(-1, 3)
    return coords, tri


def square_level0(n_side: int):
    """[-1,1]^2 grid of n_side^2 squares, each cut by the (0,0)-(1,1)
    diagonal into two right triangles (counter-clockwise)."""
    return rectangle_level0(n_side, n_side)


def square_mesh(n_coarse: int = 8, n_refine: int = 3) -> NestedMesh:
    """Uniform right-triangle mesh of [-1,1]^2 with (n_coarse*2^L)^2 squares."""
    c, t = square_level0(n_coarse)
    return build_hierarchy(2, c, t, n_refine)


# -------------------------------------------------------------- 2D asteroid
def asteroid_radius(theta):
    """Boundary of the 2D asteroid-shaped domain, r(t) = 1+0.1 sin3t+0.05 cos5t."""
    theta = np.asarray(theta, dtype=np.float64)
    return 1.0 + 0.1 * np.sin(3.0 * theta) + 0.05 * np.cos(5.0 * theta)


def ring_disk(K: int):
    """Unit disk: centre node plus K rings, ring k holding 6k nodes at radius
    k/K; neighbouring rings are joined by a zipper of triangles ordered by
    angle.  6K^2 triangles, 1+3K(K+1) nodes.  Returns (rho, theta, tris)."""
    rho, theta, rings = [0.0], [0.0], [[0]]
    nid = 1
    for k in range(1, K + 1):
        cnt = 6 * k
        ids = list(range(nid, nid + cnt))
        nid += cnt
        rings.append(ids)
        for j in range(cnt):
            rho.append(k / K)
            theta.append(2.0 * math.pi * j / cnt)
    tris = []
    for j in range(6):
        tris.append((0, rings[1][j], rings[1][(j + 1) % 6]))
    for k in range(1, K):
        inner, outer = rings[k], rings[k + 1]
        ni, no = len(inner), len(outer)
        i = j = 0
        while i < ni or j < no:
            a_next = 2.0 * math.pi * (i + 1) / ni
            b_next = 2.0 * math.pi * (j + 1) / no
            if j < no and (i >= ni or b_next <= a_next + 1e-12):
                tris.append((inner[i % ni], outer[j % no], outer[(j + 1) % no]))
                j += 1
            else:
                tris.append((inner[i % ni], outer[j % no], inner[(i + 1) % ni]))
                i += 1
    return np.array(rho), np.array(theta), np.array(tris, dtype=np.int32)


def asteroid_level0(K: int = 18, rotation: float = 0.0, scale: float = 1.0):
    rho, theta, tris = ring_disk(K)
    r = rho * asteroid_radius(theta) * scale
    coords = np.stack([r * np.cos(theta + rotation), r * np.sin(theta + rotation)], 1)
    return coords, tris


def asteroid_mesh(n_refine: int = 3, K: int = 18, rotation: float = 0.0,
                  scale: float = 1.0) -> NestedMesh:
    """2D asteroid-shaped nested mesh: 6K^2 level-0 triangles, refined
    ``n_refine`` times (K=18, 3 refinements: 124,416 triangles)."""
    c, t = asteroid_level0(K, rotation, scale)
    return build_hierarchy(2, c, t, n_refine)


# ------------------------------------------------------------- 3D ellipsoid
ELLIPSOID_AXES = (1.0, 0.8, 0.6)
ELLIPSOID_GRID = (18, 16, 12)


def ellipsoid_level0(grid=ELLIPSOID_GRID, axes=ELLIPSOID_AXES):
    """Octant-symmetric Kuhn triangulation of a box grid, mapped onto the
    ellipsoid.

    The grid has grid[a] cells along axis a on the normalised cube [-1,1]^3
    (even counts, so the origin is a node).  Each cube is cut into 6 tets
    that share the cube diagonal pointing away from the origin (mirrored per
    octant, so the triangulation is conforming across the octant planes).
    Nodes are mapped onto the unit ball by x -> x |x|_inf / |x|_2 and scaled
    by the semi-axes.  With grid (18,16,12) and axes (1,0.8,0.6) every cell
    edge along an axis is about 0.1 long; 20,736 tets."""
    N = np.asarray(grid, dtype=np.int64)
    assert np.all(N % 2 == 0)
    ax = [np.linspace(-1.0, 1.0, int(n) + 1) for n in N]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n2 = np.linalg.norm(p, axis=1)
    ninf = np.abs(p).max(axis=1)
    s = np.where(n2 > 0, ninf / np.where(n2 > 0, n2, 1.0), 0.0)
    coords = p * s[:, None] * np.asarray(axes)[None, :]
    stride = np.array([(N[1] + 1) * (N[2] + 1), N[2] + 1, 1], dtype=np.int64)
    I, J, K = np.meshgrid(*[np.arange(int(n)) for n in N], indexing="ij")
    cube = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    sign = np.where(cube >= (N // 2)[None, :], 1, -1)
    c0 = np.where(sign > 0, cube, cube + 1)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        v = c0.copy()
        vs = [v @ stride]
        for a in perm:
            v = v.copy()
            v[:, a] += sign[:, a]
            vs.append(v @ stride)
        tets.append(np.stack(vs, 1))
    tets = np.stack(tets, 1).reshape(-1, 4).astype(np.int32)
    return coords, tets


def ellipsoid_mesh(n_refine: int = 3, grid=ELLIPSOID_GRID,
                   axes=ELLIPSOID_AXES) -> NestedMesh:
    """3D ellipsoid nested tetrahedral mesh: 6*prod(grid) level-0 tets
    refined ``n_refine`` times (default: 20,736 -> 10,616,832 tets,
    1,814,385 nodes)."""
    c, t = ellipsoid_level0(grid, axes)
    return build_hierarchy(3, c, t, n_refine)


def cell_measures(mesh: NestedMesh) -> np.ndarray:
    """Unsigned cell areas/volumes of the finest level (geometry check)."""
    x = mesh.coords[mesh.cells]
    E = x[:, 1:, :] - x[:, :1, :]
    return np.abs(np.linalg.det(E)) / math.factorial(mesh.dim)


def centroids(mesh: NestedMesh) -> np.ndarray:
    return mesh.coords[mesh.cells].mean(axis=1)
