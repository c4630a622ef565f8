"""Pins of the oracle's 2D cells (triangles P1..P6, quadrilaterals Q_p; plane strain for the vector forms) against
closed forms, invariants and finite differences.  None re-evaluates the oracle's formulas."""
import math

import numpy as np
import pytest

import fe_inputs as fi
import oracle
from tests import exact


def tri_problem(nx, p, kind, perturb=0.15, seed=2, ncomp=1, qdeg=None, **kw):
    m = fi.tri_mesh(nx, perturb=perturb, seed=seed)
    cn, nn, node_coords = fi.tri_node_map(m.cell_vert, m.nvert, p)
    pb = oracle.Problem(oracle.TRI, m.coords, m.cell_vert, p, cn, nn, kind, ncomp=ncomp,
                        qdeg=qdeg if qdeg is not None else 2 * p, **kw)
    return pb, m, node_coords(m.coords)


def quad_problem(nx, p, kind, perturb=0.1, seed=1, ncomp=1, qdeg=None, **kw):
    m = fi.quad_mesh(nx, perturb=perturb, seed=seed)
    cn, nn = fi.quad_node_map(nx, p)
    pb = oracle.Problem(oracle.QUAD, m.coords, m.cell_vert, p, cn, nn, kind, ncomp=ncomp,
                        qdeg=qdeg if qdeg is not None else p + 1, **kw)
    return pb, m, quad_nodes(m, cn, p)


def quad_nodes(m, cn, p):
    n = p + 1
    s = exact.gll_nodes_np(n)
    out = np.zeros((cn.max() + 1, 3))
    X = m.coords[m.cell_vert]
    for j in range(n):
        for i in range(n):
            w = np.array([(s[i] if v & 1 else 1 - s[i]) * (s[j] if v & 2 else 1 - s[j]) for v in range(4)])
            out[cn[:, i + n * j]] = np.einsum("v,cvd->cd", w, X)
    return out


def interior_of(nodes):
    return np.all((nodes[:, :2] > 1e-12) & (nodes[:, :2] < 1 - 1e-12), axis=1)


@pytest.mark.parametrize("degree", [0, 1, 2, 4, 6, 9])
def test_tri_rule_exact_on_monomials(degree):
    pts, w = oracle.tri_rule(degree)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            ref = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * pts[:, 0] ** a * pts[:, 1] ** b).sum() - ref) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_tri_basis_nodal_in_lattice_order_and_reproduces_polynomials(p):
    lat = fi.tri_lattice(p)
    nodes = lat[:, 1:] / p
    n = lat.shape[0]
    for a in range(n):
        phi, _ = oracle.tri_basis(p, nodes[a])
        e = np.zeros(n)
        e[a] = 1.0
        np.testing.assert_allclose(phi, e, atol=1e-11)
    rng = np.random.default_rng(p)
    terms = [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]
    c = rng.standard_normal(len(terms))
    f = lambda x: sum(cc * x[0] ** i * x[1] ** j for cc, (i, j) in zip(c, terms))
    fx = lambda x: sum(cc * i * x[0] ** (i - 1) * x[1] ** j for cc, (i, j) in zip(c, terms) if i)
    fy = lambda x: sum(cc * j * x[0] ** i * x[1] ** (j - 1) for cc, (i, j) in zip(c, terms) if j)
    vals = np.array([f(x) for x in nodes])
    for _ in range(5):
        b = rng.dirichlet(np.ones(3))
        xi = b[1:]
        phi, dphi = oracle.tri_basis(p, xi)
        assert abs(phi @ vals - f(xi)) < 1e-10 * max(1.0, np.abs(vals).max())
        np.testing.assert_allclose(dphi.T @ vals, [fx(xi), fy(xi)], atol=1e-9 * max(1.0, np.abs(vals).max()))


@pytest.mark.parametrize("p", [1, 3, 5])
def test_quad_basis_kronecker_at_gll_points(p):
    n = p + 1
    s = exact.gll_nodes_np(n)
    for a in range(n * n):
        phi, _ = oracle.quad_basis(p, [s[a % n], s[a // n]])
        e = np.zeros(n * n)
        e[a] = 1.0
        np.testing.assert_allclose(phi, e, atol=1e-13)


def test_p1_triangle_element_matrices_closed_form():
    pm, m, _ = tri_problem(2, 1, oracle.MASS, qdeg=2)
    pl, _, _ = tri_problem(2, 1, oracle.LAPLACE, qdeg=2)
    for c in [0, 3, 6]:
        X = m.coords[m.cell_vert[c], :2]
        e1, e2 = X[1] - X[0], X[2] - X[0]
        area = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        np.testing.assert_allclose(pm.element_matrix(c), area / 12 * (np.ones((3, 3)) + np.eye(3)), rtol=1e-14)
        # stiffness: (b_i b_j + c_i c_j) / (4 area), b_i = y_{i+1} - y_{i+2}, c_i = x_{i+2} - x_{i+1}
        b = np.array([X[(i + 1) % 3, 1] - X[(i + 2) % 3, 1] for i in range(3)])
        cc = np.array([X[(i + 2) % 3, 0] - X[(i + 1) % 3, 0] for i in range(3)])
        np.testing.assert_allclose(pl.element_matrix(c), (np.outer(b, b) + np.outer(cc, cc)) / (4 * area), rtol=1e-13)


@pytest.mark.parametrize("cell, p", [("tri", 1), ("tri", 2), ("tri", 4), ("quad", 1), ("quad", 2), ("quad", 4)])
def test_2d_conservation_and_laplacian_null_space(cell, p):
    make = tri_problem if cell == "tri" else quad_problem
    pm, m, nodes = make(3, p, oracle.MASS)
    pl, _, _ = make(3, p, oracle.LAPLACE)
    ph, _, _ = make(3, p, oracle.HELMHOLTZ, k2=1.0)
    one = np.ones(pm.ndof)
    assert abs(pm.apply(one).sum() - 1.0) < 1e-13
    assert np.abs(pl.apply(one)).max() < 1e-13
    np.testing.assert_allclose(ph.apply(one), pm.apply(one), atol=1e-15)
    lin = 0.3 + nodes[:, :2] @ np.array([1.0, -2.0])
    y = pl.apply(lin)
    inside = interior_of(nodes)
    assert np.abs(y[inside]).max() < 1e-12 and np.abs(y[~inside]).max() > 1e-3


@pytest.mark.parametrize("cell, p", [("tri", 2), ("tri", 3), ("quad", 1), ("quad", 3)])
def test_2d_elasticity_rigid_modes_and_symmetry(cell, p):
    make = tri_problem if cell == "tri" else quad_problem
    pb, m, nodes = make(2, p, oracle.ELASTICITY, ncomp=2, lam=1.2, mu=0.8)
    for t in np.eye(2):
        assert np.abs(pb.apply(np.tile(t, (pb.nnode, 1)).ravel())).max() < 1e-13
    rot = np.stack([-nodes[:, 1], nodes[:, 0]], axis=1)
    assert np.abs(pb.apply(rot.ravel())).max() < 1e-13
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(pb.ndof), rng.standard_normal(pb.ndof)
    ax = pb.apply(x)
    assert np.abs(ax).max() > 1e-2 and abs(y @ ax - x @ pb.apply(y)) < 1e-12 * np.abs(ax).max() * pb.ndof


def rot2(theta):
    return np.array([[math.cos(theta), -math.sin(theta)], [math.sin(theta), math.cos(theta)]])


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
@pytest.mark.parametrize("cell", ["tri", "quad"])
def test_2d_hyper_rotation_and_homogeneous_deformation(law, cell):
    make = tri_problem if cell == "tri" else quad_problem
    p = 2
    pb, m, nodes = make(3, p, oracle.HYPER_RES, ncomp=2, law=law, **({"qdeg": 4} if cell == "tri" else {}))
    X = nodes[:, :2]
    R = rot2(0.7)
    assert np.abs(pb.apply((X @ R.T - X).ravel())).max() < 1e-13
    F0 = np.array([[1.1, 0.05], [-0.03, 0.92]])
    r = pb.apply((X @ (F0 - np.eye(2)).T).ravel()).reshape(-1, 2)
    inside = interior_of(nodes)
    assert np.abs(r[inside]).max() < 1e-13 and np.abs(r[~inside]).max() > 1e-4


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
@pytest.mark.parametrize("cell", ["tri", "quad"])
def test_2d_hyper_energy_gradient_jacobian_and_linearisation(law, cell):
    make = tri_problem if cell == "tri" else quad_problem
    kw = dict(ncomp=2, law=law, lam=1.3, mu=0.7)
    if cell == "tri":
        kw["qdeg"] = 4
    pr, m, nodes = make(2, 2, oracle.HYPER_RES, b=(0.2, -0.1, 0.0), **kw)
    u = fi.sinusoid_displacement(nodes, seed=3)[:, :2].ravel()
    r = pr.apply(u)
    rng = np.random.default_rng(9)
    d = rng.standard_normal(pr.ndof)
    eps = 1e-5
    fd = (pr.energy(u + eps * d) - pr.energy(u - eps * d)) / (2 * eps)
    assert abs(fd - r @ d) <= 1e-7 * max(1.0, abs(r @ d))
    pr0, _, _ = make(2, 2, oracle.HYPER_RES, **kw)
    pj, _, _ = make(2, 2, oracle.HYPER_JAC, ucoef=u, **kw)
    fdj = (pr0.apply(u + 1e-6 * d) - pr0.apply(u - 1e-6 * d)) / 2e-6
    jd = pj.apply(d)
    assert np.linalg.norm(fdj - jd) <= 1e-7 * np.linalg.norm(jd)
    pz, _, _ = make(2, 2, oracle.HYPER_JAC, ucoef=np.zeros(pr.ndof), **kw)
    kwe = {k: v for k, v in kw.items() if k != "law"}
    pe, _, _ = make(2, 2, oracle.ELASTICITY, **kwe)
    np.testing.assert_allclose(pz.apply(d), pe.apply(d), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("kind, law", [("elasticity", oracle.SVK), ("hyper_res", oracle.SVK),
                                       ("hyper_res", oracle.NEOHOOKE)])
def test_plane_strain_is_the_z_invariant_3d_problem(p, kind, law):
    """Plane strain pinned to the 3D oracle: the quad mesh extruded one unit in z as hexahedra, with the in-plane
    displacement (u1, u2, 0) at every z-level, gives residuals whose sums over each column of z-nodes equal the
    quad residual (in-plane components) and vanish (z component). The z-invariant test function is the sum of the
    column's z basis functions, so the 3D weak form reduces to the 2D one times the unit thickness."""
    from tests.problems import quad_case

    q = quad_case(3, p, ncomp=2, seed=4)
    nq, nvq = q["nnode"], q["coords"].shape[0]
    n = p + 1
    # extruded mesh: vertex v + nvq * k at height k, hex local vertex a + 2b + 4c over quad local vertex a + 2b
    coords = np.vstack([np.column_stack([q["coords"][:, :2], np.full(nvq, float(k))]) for k in (0, 1)])
    cv = np.hstack([q["cell_vert"], q["cell_vert"] + nvq]).astype(np.int32)
    # hex node (quad node, z-level k): quad node + nq * k; local hex node aq + n^2 * k
    cn = np.hstack([q["cell_node"] + nq * k for k in range(n)]).astype(np.int32)
    u2 = fi.sinusoid_displacement(q["nodes"], seed=5)[:, :2]
    u3 = np.zeros((nq * n, 3))
    for k in range(n):
        u3[nq * k:nq * (k + 1), :2] = u2
    kw = dict(lam=1.1, mu=0.7, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.05, -0.02, 0.0)
    okind = {"elasticity": oracle.ELASTICITY, "hyper_res": oracle.HYPER_RES}[kind]
    r2 = oracle.Problem(oracle.QUAD, q["coords"], q["cell_vert"], p, q["cell_node"], nq, okind, ncomp=2,
                        qdeg=p + 1, **kw).apply(u2.ravel()).reshape(-1, 2)
    r3 = oracle.Problem(oracle.HEX, coords, cv, p, cn, nq * n, okind, ncomp=3, qdeg=p + 1,
                        **kw).apply(u3.ravel()).reshape(n, nq, 3).sum(axis=0)
    scale = np.abs(r2).max()
    assert np.abs(r3[:, :2] - r2).max() <= 1e-12 * scale
    assert np.abs(r3[:, 2]).max() <= 1e-12 * scale
