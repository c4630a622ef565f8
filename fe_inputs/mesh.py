"""Synthetic meshes and cell maps.

Conventions (shared by every consumer of these arrays):

* Vertex coordinates are ``float64 [nvert][3]``.
* Tetrahedron local vertices 0..3 map to reference vertices (0,0,0), (1,0,0),
  (0,1,0), (0,0,1); every generated tetrahedron is positively oriented.
* Hexahedron local vertex ``a + 2b + 4c`` (a, b, c in {0, 1}) maps to the
  reference corner (a, b, c) of [0,1]^3.
* P2 tetrahedron local nodes: 0..3 are the vertices, 4..9 the midpoints of
  the edges (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).
* Q_p hexahedron local node ``i + n*j + n*n*k`` (n = p + 1) is the tensor
  node (i, j, k); node numbering is lexicographic on the global
  (nx*p + 1)^3 grid, so neighbouring cells share face, edge and vertex nodes.
* A vector field with ncomp components stores dof ``ncomp*node + c``.
"""
from dataclasses import dataclass
import numpy as np

from .rng import uniform, splitmix64

# Axis permutations of the Kuhn (Freudenthal) split of a box into 6 tets.
_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
_P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


@dataclass
class TetMesh:
    coords: np.ndarray     # float64 [nvert][3]
    cell_vert: np.ndarray  # int32 [ncell][4]
    nx: int
    h: float

    @property
    def ncell(self):
        return self.cell_vert.shape[0]

    @property
    def nvert(self):
        return self.coords.shape[0]


@dataclass
class HexMesh:
    coords: np.ndarray     # float64 [nvert][3]
    cell_vert: np.ndarray  # int32 [ncell][8]
    nx: int
    h: float

    @property
    def ncell(self):
        return self.cell_vert.shape[0]

    @property
    def nvert(self):
        return self.coords.shape[0]


def _grid_vertices(nx, perturb, seed):
    m = nx + 1
    h = 1.0 / nx
    k, j, i = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1).astype(np.float64)
    if perturb > 0.0:
        ii, jj, kk = i.ravel(), j.ravel(), k.ravel()
        interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < nx) & (kk > 0) & (kk < nx)
        shift = uniform(seed, 0x5E57, 3 * coords.shape[0], -perturb * h, perturb * h).reshape(-1, 3)
        coords[interior] += shift[interior]
    return coords, h


def kuhn_tet_mesh(nx, perturb=0.0, seed=0):
    """Unit cube as nx^3 boxes, each split into 6 tetrahedra sharing the main diagonal.

    Tet (box, perm) has vertices v0, v0+e_p0, v0+e_p0+e_p1, v0+(1,1,1); odd
    permutations swap local vertices 1 and 2 so that every tet has a positive
    Jacobian determinant.  ``perturb`` moves interior vertices by independent
    uniform shifts of at most ``perturb*h`` per coordinate (seeded).
    """
    coords, h = _grid_vertices(nx, perturb, seed)
    m = nx + 1
    k, j, i = np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)  # [nbox][3], x fastest

    def vid(ijk):
        return ijk[:, 0] + m * (ijk[:, 1] + m * ijk[:, 2])

    cells = np.empty((base.shape[0], 6, 4), dtype=np.int64)
    eye = np.eye(3, dtype=np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        p1 = base + eye[perm[0]]
        p2 = p1 + eye[perm[1]]
        p3 = base + 1
        v = [vid(base), vid(p1), vid(p2), vid(p3)]
        # Sign of the permutation: odd permutations swap local vertices 1 and 2.
        inversions = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        if inversions % 2 == 1:
            v[1], v[2] = v[2], v[1]
        cells[:, t, :] = np.stack(v, axis=1)
    return TetMesh(coords=coords, cell_vert=cells.reshape(-1, 4).astype(np.int32), nx=nx, h=h)


def hex_box_mesh(nx, perturb=0.1, seed=1):
    """Unit cube as nx^3 hexahedra; interior vertices shifted by U[-perturb*h, perturb*h]^3."""
    coords, h = _grid_vertices(nx, perturb, seed)
    m = nx + 1
    k, j, i = np.meshgrid(np.arange(nx), np.arange(nx), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    cv = np.empty((i.size, 8), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                cv[:, a + 2 * b + 4 * c] = (i + a) + m * ((j + b) + m * (k + c))
    return HexMesh(coords=coords, cell_vert=cv.astype(np.int32), nx=nx, h=h)


def hex_slab_mesh(nx, nz_total, z0, nz, perturb=0.1, seed=1):
    """Layers z0 .. z0+nz-1 of the box [0,1]^2 x [0, nz_total/nx] meshed by nx * nx * nz_total hexahedra of side
    h = 1/nx (one part of a z-slab partition).

    Vertices and cells are numbered lexicographically within the slab.  Every vertex interior to the whole box is
    shifted by U[-perturb*h, perturb*h]^3 drawn at its index in the whole box's lexicographic numbering, so two
    slabs that share a vertex plane agree on it, and the single slab (nz_total = nz = nx, z0 = 0) is
    hex_box_mesh(nx, perturb, seed).
    """
    m = nx + 1
    h = 1.0 / nx
    k, j, i = np.meshgrid(np.arange(z0, z0 + nz + 1), np.arange(m), np.arange(m), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    coords = np.stack([i * h, j * h, k * h], axis=1).astype(np.float64)
    if perturb > 0.0:
        interior = (i > 0) & (i < nx) & (j > 0) & (j < nx) & (k > 0) & (k < nz_total)
        first = m * m * z0  # the slab's vertices are consecutive in the whole box's numbering
        shift = uniform(seed, 0x5E57, 3 * coords.shape[0], -perturb * h, perturb * h, start=3 * first).reshape(-1, 3)
        coords[interior] += shift[interior]
    kc, jc, ic = np.meshgrid(np.arange(nz), np.arange(nx), np.arange(nx), indexing="ij")
    ic, jc, kc = ic.ravel(), jc.ravel(), kc.ravel()
    cv = np.empty((ic.size, 8), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                cv[:, a + 2 * b + 4 * c] = (ic + a) + m * ((jc + b) + m * (kc + c))
    return HexMesh(coords=coords, cell_vert=cv.astype(np.int32), nx=nx, h=h)


def hex_node_map(nx, p, nz=None):
    """Cell -> node map of continuous Q_p on a structured hex mesh of nx * nx * nz cells (nz = nx by default).

    Returns (cell_node int32 [ncell][(p+1)^3], nnode).  Local node
    i + n*j + n*n*k of cell (ci, cj, ck) is grid node
    (p*ci + i, p*cj + j, p*ck + k) on the (nx*p + 1)^2 (nz*p + 1) lattice, numbered lexicographically.
    """
    n = p + 1
    m = nx * p + 1
    nz = nx if nz is None else nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(nx), np.arange(nx), indexing="ij")
    i, j, k = i.ravel().astype(np.int64), j.ravel().astype(np.int64), k.ravel().astype(np.int64)
    lk, lj, li = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    li, lj, lk = li.ravel(), lj.ravel(), lk.ravel()
    I = p * i[:, None] + li[None, :]
    J = p * j[:, None] + lj[None, :]
    K = p * k[:, None] + lk[None, :]
    node = I + m * (J + m * K)
    return node.astype(np.int32), m * m * (nz * p + 1)


def p2_node_map(cell_vert, nvert):
    """Cell -> node map of continuous P2 on a tet mesh.

    Nodes 0..nvert-1 are the mesh vertices; edge nodes follow, numbered by the
    sorted (min, max) vertex pair of each edge.  Returns (cell_node int32
    [ncell][10], nnode, edges int64 [nedge][2]).
    """
    cv = cell_vert.astype(np.int64)
    a = np.stack([cv[:, e[0]] for e in _P2_EDGES], axis=1)
    b = np.stack([cv[:, e[1]] for e in _P2_EDGES], axis=1)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = (lo * nvert + hi).ravel()
    uniq, inv = np.unique(key, return_inverse=True)
    edges = np.stack([uniq // nvert, uniq % nvert], axis=1)
    enode = nvert + inv.reshape(-1, 6)
    cell_node = np.concatenate([cv, enode], axis=1).astype(np.int32)
    return cell_node, nvert + uniq.size, edges


def p2_node_coords(coords, edges):
    """Positions of P2 nodes: vertices, then the midpoints of ``edges``."""
    mid = 0.5 * (coords[edges[:, 0]] + coords[edges[:, 1]])
    return np.concatenate([coords, mid], axis=0)


@dataclass
class PlaneMesh:
    """A 2D mesh of the unit square; coordinates carry a zero third component."""
    coords: np.ndarray     # float64 [nvert][3], z = 0
    cell_vert: np.ndarray  # int32 [ncell][3] (triangles) or [ncell][4] (quadrilaterals)
    nx: int
    h: float

    @property
    def ncell(self):
        return self.cell_vert.shape[0]

    @property
    def nvert(self):
        return self.coords.shape[0]


def _grid_vertices_2d(nx, perturb, seed):
    m = nx + 1
    h = 1.0 / nx
    j, i = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    coords = np.stack([i.ravel() * h, j.ravel() * h, np.zeros(m * m)], axis=1).astype(np.float64)
    if perturb > 0.0:
        ii, jj = i.ravel(), j.ravel()
        interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < nx)
        shift = uniform(seed, 0x5E52, 2 * coords.shape[0], -perturb * h, perturb * h).reshape(-1, 2)
        coords[interior, :2] += shift[interior]
    return coords, h


def quad_mesh(nx, perturb=0.1, seed=1):
    """Unit square as nx^2 quadrilaterals (local vertex v at corner (v & 1, v >> 1 & 1)); interior vertices shifted
    by U[-perturb*h, perturb*h]^2."""
    coords, h = _grid_vertices_2d(nx, perturb, seed)
    m = nx + 1
    j, i = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    i, j = i.ravel(), j.ravel()
    cv = np.stack([(i + di) + m * (j + dj) for dj in (0, 1) for di in (0, 1)], axis=1)
    return PlaneMesh(coords=coords, cell_vert=cv.astype(np.int32), nx=nx, h=h)


def tri_mesh(nx, perturb=0.0, seed=0):
    """Unit square as nx^2 boxes split along the (0,0)-(1,1) diagonal into 2 triangles each, counter-clockwise;
    interior vertices shifted by U[-perturb*h, perturb*h]^2."""
    coords, h = _grid_vertices_2d(nx, perturb, seed)
    m = nx + 1
    j, i = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00, v10, v01, v11 = i + m * j, i + 1 + m * j, i + m * (j + 1), i + 1 + m * (j + 1)
    cells = np.stack([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], axis=1).reshape(-1, 3)
    return PlaneMesh(coords=coords, cell_vert=cells.astype(np.int32), nx=nx, h=h)


def quad_node_map(nx, p):
    """Cell -> node map of continuous Q_p on an nx^2 structured quad mesh.  Local node i + n*j of cell (ci, cj) is
    global grid node (p*ci + i, p*cj + j) on the (nx*p + 1)^2 lattice."""
    n = p + 1
    m = nx * p + 1
    j, i = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
    i, j = i.ravel().astype(np.int64), j.ravel().astype(np.int64)
    lj, li = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    li, lj = li.ravel(), lj.ravel()
    node = (p * i[:, None] + li[None, :]) + m * (p * j[:, None] + lj[None, :])
    return node.astype(np.int32), m * m


def tri_lattice(k):
    """Barycentric lattice of P_k on a triangle, in local node order: points (i, j)/k with i + j <= k, i fastest,
    then j.  Returns int [nloc][3] weights (b0, b1, b2) = (k - i - j, i, j)."""
    return np.array([(k - i - j, i, j) for j in range(k + 1) for i in range(k + 1 - j)], dtype=np.int64)


def tri_node_map(cell_vert, nvert, k):
    """Cell -> node map of continuous P_k on a triangle mesh, local nodes in `tri_lattice` order.  A lattice point is
    the same node in every cell that contains it (keyed by the global vertices of its support and its weights on
    them); nodes 0..nvert-1 are the vertices, the others follow in sorted key order.  Returns (cell_node, nnode,
    node_coords_fn)."""
    cv = cell_vert.astype(np.int64)
    ncell = cv.shape[0]
    lat = tri_lattice(k)
    nloc = lat.shape[0]
    gv = cv[:, None, :].repeat(nloc, axis=1)
    w = np.broadcast_to(lat[None, :, :], gv.shape)
    vkey = np.where(w > 0, gv, np.int64(-1))
    order = np.argsort(np.where(vkey < 0, np.iinfo(np.int64).max, vkey), axis=2, kind="stable")
    vs = np.take_along_axis(vkey, order, axis=2)
    ws = np.take_along_axis(w, order, axis=2)
    keys = np.concatenate([vs, ws], axis=2).reshape(-1, 6)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    is_vertex = uniq[:, 3] == k
    node_of_key = np.empty(uniq.shape[0], dtype=np.int64)
    node_of_key[is_vertex] = uniq[is_vertex, 0]
    nonv = np.flatnonzero(~is_vertex)
    node_of_key[nonv] = nvert + np.arange(nonv.size)
    cell_node = node_of_key[inv].reshape(ncell, nloc).astype(np.int32)
    nnode = nvert + nonv.size

    def node_coords(coords):
        out = np.zeros((nnode, 3))
        out[node_of_key[inv].reshape(ncell, nloc)] = np.einsum("ls,csd->cld", lat / k, coords[cv])
        return out

    return cell_node, nnode, node_coords


def pk_lattice(k):
    """Barycentric lattice of P_k on a tet, in local node order: points (i, j, l)/k with i + j + l <= k, i fastest,
    then j, then l.  Returns int [nloc][4] weights (b0, b1, b2, b3), b_s = k * (barycentric coordinate of vertex s),
    vertex 0 at the origin and vertex e + 1 at the unit vector e."""
    pts = []
    for l in range(k + 1):
        for j in range(k + 1 - l):
            for i in range(k + 1 - l - j):
                pts.append((k - i - j - l, i, j, l))
    return np.array(pts, dtype=np.int64)


def pk_node_map(cell_vert, nvert, k):
    """Cell -> node map of continuous P_k (k >= 3) on a tet mesh, local nodes in `pk_lattice` order.

    A lattice point is identified across cells by the global vertices of its support and its weights on them
    (an edge, face or interior point is the same node in every cell that contains it, whatever the local vertex
    order).  Nodes 0..nvert-1 are the mesh vertices; the other nodes follow in sorted key order.  Returns
    (cell_node int32 [ncell][nloc], nnode, node_coords_fn) where node_coords_fn(coords) gives the node positions.
    """
    cv = cell_vert.astype(np.int64)
    ncell = cv.shape[0]
    lat = pk_lattice(k)
    nloc = lat.shape[0]
    # per (cell, local node): support vertices sorted by global id, with their weights; padding (-1, 0)
    gv = cv[:, None, :].repeat(nloc, axis=1)                      # [ncell][nloc][4]
    w = np.broadcast_to(lat[None, :, :], gv.shape)
    vkey = np.where(w > 0, gv, np.int64(-1))
    order = np.argsort(np.where(vkey < 0, np.iinfo(np.int64).max, vkey), axis=2, kind="stable")
    vs = np.take_along_axis(vkey, order, axis=2)
    ws = np.take_along_axis(w, order, axis=2)
    keys = np.concatenate([vs, ws], axis=2).reshape(-1, 8)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    is_vertex = (uniq[:, 4] == k)                                  # a single support vertex with the full weight
    node_of_key = np.empty(uniq.shape[0], dtype=np.int64)
    node_of_key[is_vertex] = uniq[is_vertex, 0]
    nonv = np.flatnonzero(~is_vertex)
    node_of_key[nonv] = nvert + np.arange(nonv.size)
    cell_node = node_of_key[inv].reshape(ncell, nloc).astype(np.int32)
    nnode = nvert + nonv.size

    def node_coords(coords):
        out = np.zeros((nnode, 3))
        out[node_of_key[inv].reshape(ncell, nloc)] = np.einsum("ls,csd->cld", lat / k, coords[cv])
        return out

    return cell_node, nnode, node_coords


def shuffle_mesh(cell_vert, cell_node, nnode, seed, shuffle_cells=True, shuffle_nodes=True):
    """Seeded random relabelling of cells and nodes (an unstructured ordering).

    Returns (cell_vert, cell_node, node_perm) where node ``old`` is renamed
    ``node_perm[old]``.  Vertex maps are permuted with the cells only.
    """
    ncell = cell_vert.shape[0]
    cv, cn = cell_vert, cell_node
    if shuffle_cells:
        order = np.argsort(splitmix64(seed, 0xCE11, ncell), kind="stable")
        cv, cn = cv[order], cn[order]
    node_perm = np.arange(nnode, dtype=np.int64)
    if shuffle_nodes:
        node_perm = np.argsort(np.argsort(splitmix64(seed, 0x40DE, nnode), kind="stable"), kind="stable")
        cn = node_perm[cn.astype(np.int64)].astype(np.int32)
    return np.ascontiguousarray(cv), np.ascontiguousarray(cn), node_perm
