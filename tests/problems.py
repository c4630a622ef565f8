"""Shared problem builders: one set of seeded inputs, handed to both the oracle and the library."""
import numpy as np

import fe_inputs as fi
import oracle

KIND_NAMES = {"mass": 0, "laplace": 1, "helmholtz": 2, "elasticity": 3, "hyper_res": 4, "hyper_jac": 5}


def hex_node_coords(m, cn, p):
    """Physical positions of the Q_p nodes: trilinear image of numpy-derived GLL points."""
    from tests import exact

    n = p + 1
    s = exact.gll_nodes_np(n)
    out = np.zeros((cn.max() + 1, 3))
    X = m.coords[m.cell_vert]  # [ncell][8][3]
    for k in range(n):
        for j in range(n):
            for i in range(n):
                a = i + n * j + n * n * k
                xi = (s[i], s[j], s[k])
                w = np.array([(xi[0] if v & 1 else 1 - xi[0]) * (xi[1] if v & 2 else 1 - xi[1]) *
                              (xi[2] if v & 4 else 1 - xi[2]) for v in range(8)])
                out[cn[:, a]] = np.einsum("v,cvd->cd", w, X)
    return out


def hex_case(nx, p, perturb=0.1, seed=1, shuffle=False, ncomp=1):
    mesh = fi.hex_box_mesh(nx, perturb=perturb, seed=seed)
    cell_node, nnode = fi.hex_node_map(nx, p)
    nodes = hex_node_coords(mesh, cell_node, p) if ncomp == 3 else None
    cv = mesh.cell_vert
    if shuffle:
        cv, cell_node, perm = fi.shuffle_mesh(cv, cell_node, nnode, seed=seed + 100)
        if nodes is not None:
            inv = np.empty_like(perm)
            inv[perm] = np.arange(perm.size)
            nodes = nodes[inv]
    return dict(cell_type=8, coords=mesh.coords, cell_vert=cv, degree=p, cell_node=cell_node, nnode=nnode,
                ncomp=ncomp, nodes=nodes)


def tet_case(nx, p, ncomp=1, perturb=0.0, seed=0, shuffle=False):
    mesh = fi.kuhn_tet_mesh(nx, perturb=perturb, seed=seed)
    if p == 1:
        cn, nnode, nodes = mesh.cell_vert, mesh.nvert, mesh.coords
    elif p >= 3:
        cn, nnode, node_coords = fi.pk_node_map(mesh.cell_vert, mesh.nvert, p)
        nodes = node_coords(mesh.coords)
    else:
        cn, nnode, edges = fi.p2_node_map(mesh.cell_vert, mesh.nvert)
        nodes = fi.p2_node_coords(mesh.coords, edges)
    cv = mesh.cell_vert
    if shuffle:
        cv, cn, perm = fi.shuffle_mesh(cv, cn, nnode, seed=seed + 100)
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        nodes = nodes[inv]
    return dict(cell_type=4, coords=mesh.coords, cell_vert=cv, degree=p, cell_node=cn, nnode=nnode, ncomp=ncomp,
                nodes=nodes)


def quad_case(nx, p, ncomp=1, perturb=0.1, seed=1):
    """Perturbed unit-square quads with the structured Q_p map; node positions for vector inputs."""
    mesh = fi.quad_mesh(nx, perturb=perturb, seed=seed)
    cn, nnode = fi.quad_node_map(nx, p)
    nodes = None
    if ncomp == 2:
        from tests import exact

        n = p + 1
        s = exact.gll_nodes_np(n)
        nodes = np.zeros((nnode, 3))
        X = mesh.coords[mesh.cell_vert]
        for j in range(n):
            for i in range(n):
                w = np.array([(s[i] if v & 1 else 1 - s[i]) * (s[j] if v & 2 else 1 - s[j]) for v in range(4)])
                nodes[cn[:, i + n * j]] = np.einsum("v,cvd->cd", w, X)
    return dict(cell_type=40, coords=mesh.coords, cell_vert=mesh.cell_vert, degree=p, cell_node=cn, nnode=nnode,
                ncomp=ncomp, nodes=nodes)


def tri_case(nx, p, ncomp=1, perturb=0.15, seed=2):
    mesh = fi.tri_mesh(nx, perturb=perturb, seed=seed)
    cn, nnode, node_coords = fi.tri_node_map(mesh.cell_vert, mesh.nvert, p)
    return dict(cell_type=3, coords=mesh.coords, cell_vert=mesh.cell_vert, degree=p, cell_node=cn, nnode=nnode,
                ncomp=ncomp, nodes=node_coords(mesh.coords))


def oracle_problem(case, kind, qdeg=None, **kw):
    if qdeg is None:
        if case["cell_type"] in (8, 40):
            qdeg = case["degree"] + 1
        else:
            p = case["degree"]
            qdeg = (max(4, 2 * p) if p > 2 else 4) if kind in ("hyper_res", "hyper_jac") else 2 * p
    return oracle.Problem(case["cell_type"], case["coords"], case["cell_vert"], case["degree"], case["cell_node"],
                          case["nnode"], KIND_NAMES[kind], ncomp=case["ncomp"], qdeg=qdeg, **kw)


def cells_touching(cell_node, dofs, ncomp=1):
    """Cells whose map contains any node of the given dofs (for sampled full-size parity)."""
    nodes = np.unique(np.asarray(dofs) // ncomp)
    mask = np.isin(cell_node, nodes).any(axis=1)
    return np.nonzero(mask)[0]


def assembled_dense(pb, case):
    """The global matrix assembled from the oracle's element matrices (local dofs a * ncomp + c): the same matrix
    as pb.dense(), one oracle call per cell instead of one per dof."""
    nc, cn = case["ncomp"], case["cell_node"]
    n = case["nnode"] * nc
    A = np.zeros((n, n))
    for cell in range(cn.shape[0]):
        Ae = pb.element_matrix(cell)
        dofs = (nc * cn[cell][:, None] + np.arange(nc)[None, :]).ravel()
        A[np.ix_(dofs, dofs)] += Ae
    return A
