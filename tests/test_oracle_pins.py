"""Pins of the FP64 oracle against facts fixed outside it.

Each test compares the oracle with a closed form, an independent library
routine (numpy polynomials / linear algebra), a conservation law or an
invariant of the forms in arXiv 1903.08243 (Supplementary material), or a
finite-difference derivative.  None of them re-evaluates the oracle's own
formulas.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as L

import oracle
import fe_inputs as fi
from tests import exact
from tests.problems import hex_node_coords

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- quadrature

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 12])
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    x, w = oracle.gauss_legendre(n)
    t, wt = L.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (1 + t), rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wt, rtol=0, atol=1e-15)
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-15


@pytest.mark.parametrize("alpha", [1, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6])
def test_gauss_jacobi_exact_on_beta_integrals(n, alpha):
    x, w = oracle.gauss_jacobi(n, alpha)
    for k in range(2 * n):
        # int_0^1 x^k (1-x)^alpha dx = k! alpha! / (k + alpha + 1)!
        exact_v = math.factorial(k) * math.factorial(alpha) / math.factorial(k + alpha + 1)
        assert abs(np.dot(w, x ** k) - exact_v) < 1e-15
    # n points cannot integrate degree 2n exactly (it is a Gauss rule, not more)
    exact_v = math.factorial(2 * n) * math.factorial(alpha) / math.factorial(2 * n + alpha + 1)
    assert abs(np.dot(w, x ** (2 * n)) - exact_v) > 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 9])
def test_gll_nodes_match_numpy(n):
    np.testing.assert_allclose(oracle.gll_nodes(n), exact.gll_nodes_np(n), rtol=0, atol=2e-15)


@pytest.mark.parametrize("degree", [1, 2, 3, 4, 5, 6])
def test_tet_rule_exact_on_monomials(degree):
    pts, w = oracle.tet_rule(degree)
    assert np.all(w > 0)
    assert np.all(pts >= 0) and np.all(pts.sum(axis=1) <= 1)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                ex = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.dot(w, pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(got - ex) < 1e-16, (a, b, c)


# ---------------------------------------------------------------- bases

def test_local_dof_counts_match_table2():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table2_local_dofs.txt")) if l[0] != "#"]
    for cell, p, D in rows:
        p, D = int(p), int(D)
        if cell == "tet" and p <= 2:
            phi, _ = oracle.tet_basis(p, [0.1, 0.2, 0.3])
            assert phi.size == D
        if cell == "hex":
            phi, _ = oracle.hex_basis(p, [0.1, 0.2, 0.3])
            assert phi.size == D ** 3


def _tet_nodes(p):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    if p == 1:
        return v
    mids = [0.5 * (v[a] + v[b]) for a, b in exact.P2_EDGES]
    return np.vstack([v, mids])


@pytest.mark.parametrize("p", [1, 2])
def test_tet_basis_kronecker_and_reproduction(p):
    nodes = _tet_nodes(p)
    for i, xn in enumerate(nodes):
        phi, _ = oracle.tet_basis(p, xn)
        np.testing.assert_allclose(phi, np.eye(len(nodes))[i], atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(10):
        xi = rng.dirichlet(np.ones(4))[1:]
        phi, dphi = oracle.tet_basis(p, xi)
        assert abs(phi.sum() - 1) < 1e-15
        np.testing.assert_allclose(dphi.sum(axis=0), 0, atol=1e-14)
        # reproduces every polynomial of degree <= p, with its gradient
        f = lambda x: 0.3 + x[0] - 2 * x[1] + 0.5 * x[2] + (p == 2) * (x[0] * x[1] - x[2] ** 2 + 0.7 * x[0] ** 2)
        g = lambda x: np.array([1 + (p == 2) * (x[1] + 1.4 * x[0]), -2 + (p == 2) * x[0], 0.5 - (p == 2) * 2 * x[2]])
        fv = np.array([f(x) for x in nodes])
        assert abs(phi @ fv - f(xi)) < 1e-14
        np.testing.assert_allclose(dphi.T @ fv, g(xi), atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_hex_basis_kronecker_at_gll_tensor_nodes(p):
    n = p + 1
    s = exact.gll_nodes_np(n)
    rng = np.random.default_rng(p)
    for a in rng.choice(n ** 3, size=min(20, n ** 3), replace=False):
        i, j, k = a % n, (a // n) % n, a // (n * n)
        phi, dphi = oracle.hex_basis(p, [s[i], s[j], s[k]])
        e = np.zeros(n ** 3)
        e[a] = 1
        np.testing.assert_allclose(phi, e, atol=1e-13)
    xi = rng.random(3)
    phi, dphi = oracle.hex_basis(p, xi)
    assert abs(phi.sum() - 1) < 1e-13
    np.testing.assert_allclose(dphi.sum(axis=0), 0, atol=1e-11)


# ---------------------------------------------------------------- helpers

def tet_problem(nx, p, kind, perturb=0.0, seed=0, ncomp=1, qdeg=None, **kw):
    m = fi.kuhn_tet_mesh(nx, perturb=perturb, seed=seed)
    if p == 1:
        cn, nnode = m.cell_vert, m.nvert
        nodes = m.coords
    elif p >= 3:
        cn, nnode, node_coords = fi.pk_node_map(m.cell_vert, m.nvert, p)
        nodes = node_coords(m.coords)
    else:
        cn, nnode, edges = fi.p2_node_map(m.cell_vert, m.nvert)
        nodes = fi.p2_node_coords(m.coords, edges)
    pb = oracle.Problem(oracle.TET, m.coords, m.cell_vert, p, cn, nnode, kind, ncomp=ncomp,
                        qdeg=qdeg if qdeg is not None else max(2 * p, 2), **kw)
    return pb, m, nodes


def hex_problem(nx, p, kind, perturb=0.1, seed=1, **kw):
    m = fi.hex_box_mesh(nx, perturb=perturb, seed=seed)
    cn, nnode = fi.hex_node_map(nx, p)
    pb = oracle.Problem(oracle.HEX, m.coords, m.cell_vert, p, cn, nnode, kind, **kw)
    return pb, m, cn


# ---------------------------------------------------------------- mass / Laplace / Helmholtz

def test_p1_tet_mass_element_matrix_closed_form():
    pb, m, _ = tet_problem(2, 1, oracle.MASS, perturb=0.15, seed=7)
    for c in [0, 5, 17, 40]:
        X = m.coords[m.cell_vert[c]]
        vol = abs(np.linalg.det(np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]]))) / 6
        np.testing.assert_allclose(pb.element_matrix(c), vol / 20 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-14)


def test_p1_tet_mass_of_one_on_kuhn_mesh():
    nx = 8
    pb, m, _ = tet_problem(nx, 1, oracle.MASS)
    y = pb.apply(np.ones(pb.ndof))
    assert abs(y.sum() - 1.0) < 1e-14
    v = np.arange(m.nvert)
    i, j, k = v % (nx + 1), (v // (nx + 1)) % (nx + 1), v // (nx + 1) ** 2
    interior = (i > 0) & (i < nx) & (j > 0) & (j < nx) & (k > 0) & (k < nx)
    # each interior vertex lies in 24 tets of volume h^3/6, a quarter of each
    np.testing.assert_allclose(y[interior], (1.0 / nx) ** 3, rtol=1e-13)


@pytest.mark.parametrize("p", [1, 2])
@pytest.mark.parametrize("kind", ["mass", "grad"])
def test_tet_element_matrices_exact(p, kind):
    k = oracle.MASS if kind == "mass" else oracle.LAPLACE
    pb, m, _ = tet_problem(2, p, k, perturb=0.2, seed=3, qdeg=2 * p)
    for c in [1, 11, 30]:
        M, I, vol = exact.tet_exact(m.coords[m.cell_vert[c]], p)
        ref = M if kind == "mass" else np.einsum("abjj->ab", I)
        np.testing.assert_allclose(pb.element_matrix(c), ref, rtol=1e-12, atol=1e-15 * abs(ref).max())


@pytest.mark.parametrize("p", [1, 2, 3, 5])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
def test_affine_hex_element_matrices_exact(p, kind):
    """On an affine (sheared, stretched) hex the Q_p matrices factor into exact 1D integrals."""
    A = np.array([[0.9, 0.2, 0.1], [-0.1, 1.3, 0.25], [0.05, -0.3, 0.7]])
    b = np.array([0.3, -0.2, 0.1])
    corners = np.array([[(v & 1), (v >> 1) & 1, (v >> 2) & 1] for v in range(8)], dtype=float)
    coords = corners @ A.T + b
    n = p + 1
    cn = np.arange(n ** 3, dtype=np.int32)[None, :]
    kd = {"mass": oracle.MASS, "laplace": oracle.LAPLACE, "helmholtz": oracle.HELMHOLTZ}[kind]
    pb = oracle.Problem(oracle.HEX, coords, np.arange(8)[None, :], p, cn, n ** 3, kd, k2=0.7)
    ref = exact.affine_hex_matrices(p, A, kind, k2=0.7)
    np.testing.assert_allclose(pb.element_matrix(0), ref, rtol=1e-11, atol=1e-13 * abs(ref).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_perturbed_hex_conservation_and_null_spaces(p):
    nx = 3
    pb_m, m, cn = hex_problem(nx, p, oracle.MASS)
    pb_l, _, _ = hex_problem(nx, p, oracle.LAPLACE)
    pb_h, _, _ = hex_problem(nx, p, oracle.HELMHOLTZ)
    one = np.ones(pb_m.ndof)
    ym = pb_m.apply(one)
    # Gauss with p+1 points integrates det J (degree <= 2 per direction) exactly
    assert abs(ym.sum() - 1.0) < 1e-13
    np.testing.assert_allclose(pb_l.apply(one), 0, atol=1e-13)
    np.testing.assert_allclose(pb_h.apply(one), ym, atol=1e-14)
    # linear field: zero Laplacian action at interior nodes (exact quadrature for p >= 1)
    X = hex_node_coords(m, cn, p)
    lin = 0.3 + X @ np.array([1.0, -2.0, 0.5])
    yl = pb_l.apply(lin)
    M = nx * p + 1
    v = np.arange(M ** 3)
    i, j, k = v % M, (v // M) % M, v // (M * M)
    interior = (i > 0) & (i < M - 1) & (j > 0) & (j < M - 1) & (k > 0) & (k < M - 1)
    assert np.abs(yl[interior]).max() < 1e-13
    assert np.abs(yl[~interior]).max() > 1e-3  # boundary flux is not zero


def test_brute_force_dense_assembly_p1_tet():
    """Global matrix from closed-form P1 element matrices equals the oracle's action."""
    pb, m, _ = tet_problem(2, 1, oracle.MASS, perturb=0.2, seed=5)
    A = np.zeros((m.nvert, m.nvert))
    for c in range(m.ncell):
        X = m.coords[m.cell_vert[c]]
        vol = abs(np.linalg.det(np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]]))) / 6
        idx = m.cell_vert[c]
        A[np.ix_(idx, idx)] += vol / 20 * (np.ones((4, 4)) + np.eye(4))
    np.testing.assert_allclose(pb.dense(), A, rtol=1e-13, atol=1e-17)


def test_brute_force_dense_assembly_affine_hex_q2():
    """Unperturbed 2x2x2 Q2 mesh: global Helmholtz matrix from exact 1D Kronecker elements."""
    nx, p = 2, 2
    pb, m, cn = hex_problem(nx, p, oracle.HELMHOLTZ, perturb=0.0)
    Ke = exact.affine_hex_matrices(p, np.eye(3) / nx, "helmholtz")
    A = np.zeros((pb.ndof, pb.ndof))
    for c in range(m.ncell):
        A[np.ix_(cn[c], cn[c])] += Ke
    np.testing.assert_allclose(pb.dense(), A, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("case", ["tetP1mass", "tetP2lap3", "hexQ2helm", "hexQ3lap"])
def test_symmetry(case):
    rng = np.random.default_rng(1)
    if case == "tetP1mass":
        pb, _, _ = tet_problem(3, 1, oracle.MASS, perturb=0.2)
    elif case == "tetP2lap3":
        pb, _, _ = tet_problem(2, 2, oracle.LAPLACE, perturb=0.2, ncomp=3)
    elif case == "hexQ2helm":
        pb, _, _ = hex_problem(3, 2, oracle.HELMHOLTZ)
    else:
        pb, _, _ = hex_problem(2, 3, oracle.LAPLACE)
    x, y = rng.standard_normal(pb.ndof), rng.standard_normal(pb.ndof)
    a, b = x @ pb.apply(y), y @ pb.apply(x)
    assert abs(a - b) <= 1e-13 * max(abs(a), 1)


# ---------------------------------------------------------------- elasticity

def test_p2_elasticity_element_matrix_exact():
    lam, mu = 1.3, 0.8
    pb, m, _ = tet_problem(2, 2, oracle.ELASTICITY, perturb=0.2, seed=9, ncomp=3, lam=lam, mu=mu, qdeg=4)
    for c in [2, 23]:
        _, I, _ = exact.tet_exact(m.coords[m.cell_vert[c]], 2)
        n = 10
        ref = np.zeros((3 * n, 3 * n))
        for a in range(n):
            for cc in range(3):
                for b in range(n):
                    for d in range(3):
                        # sigma(phi_b e_d) : grad(phi_a e_c)
                        v = (mu * (cc == d) * np.trace(I[a, b]) + mu * I[a, b, d, cc] + lam * I[a, b, cc, d])
                        ref[3 * a + cc, 3 * b + d] = v
        np.testing.assert_allclose(pb.element_matrix(c), ref, rtol=1e-12, atol=1e-14 * abs(ref).max())


def test_p2_elasticity_rigid_modes_and_symmetry():
    pb, m, nodes = tet_problem(3, 2, oracle.ELASTICITY, perturb=0.2, seed=2, ncomp=3, lam=1.0, mu=1.0, qdeg=4)
    for t in np.eye(3):
        u = np.tile(t, (pb.nnode, 1))
        assert np.abs(pb.apply(u)).max() < 1e-14
    for w in np.eye(3):
        u = np.cross(w, nodes)  # infinitesimal rotation: in the P2 space, zero strain
        assert np.abs(pb.apply(u)).max() < 1e-13
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(pb.ndof), rng.standard_normal(pb.ndof)
    assert abs(x @ pb.apply(y) - y @ pb.apply(x)) < 1e-12


# ---------------------------------------------------------------- hyperelasticity

def _rotation(theta, axis):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(theta) * K + (1 - math.cos(theta)) * K @ K


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hyper_rigid_rotation_has_zero_residual(law):
    pb, m, nodes = tet_problem(2, 2, oracle.HYPER_RES, perturb=0.2, seed=4, ncomp=3, qdeg=4, law=law)
    R = _rotation(0.7, [1, 2, 3])
    u = nodes @ R.T - nodes
    assert np.abs(pb.apply(u)).max() < 1e-13


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hyper_residual_is_energy_gradient(law):
    b = (0.1, -0.2, 0.3)
    pb, m, nodes = tet_problem(2, 2, oracle.HYPER_RES, perturb=0.2, seed=4, ncomp=3, qdeg=4, law=law,
                               lam=1.0, mu=1.0, b=b)
    u = fi.sinusoid_displacement(nodes, seed=2).ravel()
    r = pb.apply(u)
    rng = np.random.default_rng(5)
    for _ in range(3):
        d = rng.standard_normal(pb.ndof)
        eps = 1e-5
        fd = (pb.energy(u + eps * d) - pb.energy(u - eps * d)) / (2 * eps)
        assert abs(fd - r @ d) <= 1e-7 * max(1.0, abs(r @ d)), (fd, r @ d)


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hyper_jacobian_is_residual_derivative(law):
    pbr, m, nodes = tet_problem(2, 2, oracle.HYPER_RES, perturb=0.2, seed=4, ncomp=3, qdeg=4, law=law)
    u = fi.sinusoid_displacement(nodes, seed=3).ravel()
    pbj = oracle.Problem(oracle.TET, m.coords, m.cell_vert, 2, pbr.cell_node, pbr.nnode, oracle.HYPER_JAC,
                         ncomp=3, qdeg=4, law=law, ucoef=u)
    rng = np.random.default_rng(6)
    d = rng.standard_normal(pbr.ndof)
    eps = 1e-6
    fd = (pbr.apply(u + eps * d) - pbr.apply(u - eps * d)) / (2 * eps)
    jd = pbj.apply(d)
    assert np.linalg.norm(fd - jd) <= 1e-7 * np.linalg.norm(jd)
    # the tangent has major symmetry
    e = rng.standard_normal(pbr.ndof)
    assert abs(e @ pbj.apply(d) - d @ pbj.apply(e)) < 1e-11 * abs(e @ jd)


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hyper_linearisation_at_zero_is_linear_elasticity(law):
    lam, mu = 1.7, 0.6
    pbe, m, nodes = tet_problem(2, 2, oracle.ELASTICITY, perturb=0.2, seed=8, ncomp=3, qdeg=4, lam=lam, mu=mu)
    pbj = oracle.Problem(oracle.TET, m.coords, m.cell_vert, 2, pbe.cell_node, pbe.nnode, oracle.HYPER_JAC,
                         ncomp=3, qdeg=4, law=law, lam=lam, mu=mu, ucoef=np.zeros(pbe.ndof))
    d = np.random.default_rng(7).standard_normal(pbe.ndof)
    np.testing.assert_allclose(pbj.apply(d), pbe.apply(d), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hyper_homogeneous_deformation_interior_balance(law):
    """A homogeneous deformation has constant stress: interior residuals vanish."""
    nx = 3
    pb, m, nodes = tet_problem(nx, 2, oracle.HYPER_RES, perturb=0.0, ncomp=3, qdeg=4, law=law)
    F0 = np.array([[1.1, 0.05, 0.0], [0.02, 0.95, 0.1], [0.0, -0.04, 1.05]])
    u = nodes @ (F0 - np.eye(3)).T
    r = pb.apply(u).reshape(-1, 3)
    inside = np.all((nodes > 1e-12) & (nodes < 1 - 1e-12), axis=1)
    assert np.abs(r[inside]).max() < 1e-13
    assert np.abs(r[~inside]).max() > 1e-4


# ---------------------------------------------------------------- vector forms on hexahedra

@pytest.mark.parametrize("p", [1, 2, 3])
def test_hex_elasticity_rigid_modes_and_symmetry(p):
    """Translations and infinitesimal rotations are in the Q_p space (the trilinear map is in Q_1) and have zero
    strain, so their action vanishes on a perturbed mesh; the operator is symmetric."""
    pb, m, cn = hex_problem(2, p, oracle.ELASTICITY, ncomp=3, lam=1.3, mu=0.7)
    X = hex_node_coords(m, cn, p)
    for t in np.eye(3):
        assert np.abs(pb.apply(np.tile(t, (pb.nnode, 1)).ravel())).max() < 1e-13
    for w in np.eye(3):
        assert np.abs(pb.apply(np.cross(w, X).ravel())).max() < 1e-13
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal(pb.ndof), rng.standard_normal(pb.ndof)
    ax = pb.apply(x)
    assert np.abs(ax).max() > 1e-2
    assert abs(y @ ax - x @ pb.apply(y)) < 1e-12 * np.abs(ax).max() * pb.ndof


@pytest.mark.parametrize("p", [1, 3])
def test_hex_vector_laplacian_null_space(p):
    """Constant vector fields are in the kernel; linear fields have zero action at interior nodes."""
    nx = 3
    pb, m, cn = hex_problem(nx, p, oracle.LAPLACE, ncomp=3)
    X = hex_node_coords(m, cn, p)
    assert np.abs(pb.apply(np.tile([1.0, -2.0, 0.5], pb.nnode))).max() < 1e-13
    lin = X @ np.array([[1.0, 0.2, -0.3], [0.5, -1.0, 0.1], [0.0, 0.7, 2.0]]).T + np.array([0.1, 0.2, 0.3])
    y = pb.apply(lin.ravel()).reshape(-1, 3)
    M = nx * p + 1
    v = np.arange(M ** 3)
    i, j, k = v % M, (v // M) % M, v // (M * M)
    interior = (i > 0) & (i < M - 1) & (j > 0) & (j < M - 1) & (k > 0) & (k < M - 1)
    assert np.abs(y[interior]).max() < 1e-13
    assert np.abs(y[~interior]).max() > 1e-3


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
@pytest.mark.parametrize("p", [1, 2])
def test_hex_hyper_rigid_rotation_has_zero_residual(law, p):
    pb, m, cn = hex_problem(2, p, oracle.HYPER_RES, ncomp=3, law=law)
    X = hex_node_coords(m, cn, p)
    R = _rotation(0.6, [2, -1, 1])
    assert np.abs(pb.apply((X @ R.T - X).ravel())).max() < 1e-13


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hex_hyper_homogeneous_deformation_interior_balance(law):
    """Constant F gives constant stress; Gauss with p+1 points integrates grad(phi) dx exactly on trilinear cells,
    so interior residuals vanish."""
    nx, p = 3, 2
    pb, m, cn = hex_problem(nx, p, oracle.HYPER_RES, ncomp=3, law=law)
    X = hex_node_coords(m, cn, p)
    F0 = np.array([[1.1, 0.05, 0.0], [0.02, 0.95, 0.1], [0.0, -0.04, 1.05]])
    r = pb.apply((X @ (F0 - np.eye(3)).T).ravel()).reshape(-1, 3)
    M = nx * p + 1
    v = np.arange(M ** 3)
    i, j, k = v % M, (v // M) % M, v // (M * M)
    interior = (i > 0) & (i < M - 1) & (j > 0) & (j < M - 1) & (k > 0) & (k < M - 1)
    assert np.abs(r[interior]).max() < 1e-13
    assert np.abs(r[~interior]).max() > 1e-4


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hex_hyper_residual_is_energy_gradient(law):
    pb, m, cn = hex_problem(2, 2, oracle.HYPER_RES, ncomp=3, law=law, b=(0.1, -0.2, 0.3))
    u = fi.sinusoid_displacement(hex_node_coords(m, cn, 2), seed=2).ravel()
    r = pb.apply(u)
    rng = np.random.default_rng(12)
    for _ in range(3):
        d = rng.standard_normal(pb.ndof)
        eps = 1e-5
        fd = (pb.energy(u + eps * d) - pb.energy(u - eps * d)) / (2 * eps)
        assert abs(fd - r @ d) <= 1e-7 * max(1.0, abs(r @ d)), (fd, r @ d)


@pytest.mark.parametrize("law", [oracle.SVK, oracle.NEOHOOKE])
def test_hex_hyper_jacobian_is_residual_derivative_and_linearises_to_elasticity(law):
    lam, mu = 1.4, 0.8
    pbr, m, cn = hex_problem(2, 2, oracle.HYPER_RES, ncomp=3, law=law, lam=lam, mu=mu)
    u = fi.sinusoid_displacement(hex_node_coords(m, cn, 2), seed=3).ravel()
    pbj, _, _ = hex_problem(2, 2, oracle.HYPER_JAC, ncomp=3, law=law, lam=lam, mu=mu, ucoef=u)
    rng = np.random.default_rng(13)
    d = rng.standard_normal(pbr.ndof)
    eps = 1e-6
    fd = (pbr.apply(u + eps * d) - pbr.apply(u - eps * d)) / (2 * eps)
    jd = pbj.apply(d)
    assert np.linalg.norm(fd - jd) <= 1e-7 * np.linalg.norm(jd)
    e = rng.standard_normal(pbr.ndof)
    assert abs(e @ jd - d @ pbj.apply(e)) < 1e-11 * abs(e @ jd) + 1e-12
    pb0, _, _ = hex_problem(2, 2, oracle.HYPER_JAC, ncomp=3, law=law, lam=lam, mu=mu, ucoef=np.zeros(pbr.ndof))
    pbe, _, _ = hex_problem(2, 2, oracle.ELASTICITY, ncomp=3, lam=lam, mu=mu)
    np.testing.assert_allclose(pb0.apply(d), pbe.apply(d), rtol=1e-12, atol=1e-14)


def test_elasticity_null_space_is_the_six_rigid_modes_and_clamping_removes_it():
    """The assembled P2 elasticity matrix has exactly the 6 rigid modes as its kernel (3 translations, 3
    infinitesimal rotations); replacing the rows and columns of a clamped face by the identity leaves an SPD
    matrix, which is what Dirichlet-constrained CG solves."""
    pb, m, nodes = tet_problem(2, 2, oracle.ELASTICITY, perturb=0.1, seed=9, ncomp=3, lam=1.0, mu=1.0, qdeg=4)
    A = pb.dense()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    scale = ev.max()
    assert np.sum(np.abs(ev) < 1e-10 * scale) == 6
    assert ev.min() > -1e-10 * scale
    fixed = np.flatnonzero(nodes[:, 0] < 1e-12)
    dofs = (3 * fixed[:, None] + np.arange(3)).ravel()
    R = np.ones(pb.ndof)
    R[dofs] = 0.0
    AD = R[:, None] * A * R[None, :] + np.diag(1.0 - R)
    assert np.linalg.eigvalsh(0.5 * (AD + AD.T)).min() > 1e-6 * scale


# ---------------------------------------------------------------- tets of degree 3..6

@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_tet_pk_basis_node_order_and_polynomial_reproduction(p):
    """The oracle's basis is nodal at the input generator's lattice points, in the same order, and reproduces
    every polynomial of degree p (checked against numpy evaluation)."""
    lat = fi.pk_lattice(p)
    nodes = lat[:, 1:] / p
    n = lat.shape[0]
    for a in range(n):
        phi, _ = oracle.tet_basis(p, nodes[a])
        e = np.zeros(n)
        e[a] = 1.0
        np.testing.assert_allclose(phi, e, atol=1e-11)
    rng = np.random.default_rng(p)
    terms = [(i, j, k) for i in range(p + 1) for j in range(p + 1 - i) for k in range(p + 1 - i - j)]
    coef = rng.standard_normal(len(terms))

    def f(x):
        return sum(c * x[0] ** i * x[1] ** j * x[2] ** k for c, (i, j, k) in zip(coef, terms))

    def grad(x):
        g = np.zeros(3)
        for c, (i, j, k) in zip(coef, terms):
            if i:
                g[0] += c * i * x[0] ** (i - 1) * x[1] ** j * x[2] ** k
            if j:
                g[1] += c * j * x[0] ** i * x[1] ** (j - 1) * x[2] ** k
            if k:
                g[2] += c * k * x[0] ** i * x[1] ** j * x[2] ** (k - 1)
        return g

    vals = np.array([f(x) for x in nodes])
    for _ in range(5):
        xi = rng.dirichlet(np.ones(4))[1:]
        phi, dphi = oracle.tet_basis(p, xi)
        assert abs(phi @ vals - f(xi)) < 1e-10 * max(1.0, np.abs(vals).max())
        np.testing.assert_allclose(dphi.T @ vals, grad(xi), atol=1e-9 * max(1.0, np.abs(vals).max()))


def test_tet_p3_element_matrices_exact():
    pb, m, _ = tet_problem(2, 3, oracle.MASS, perturb=0.2, seed=3, qdeg=6)
    pl, _, _ = tet_problem(2, 3, oracle.LAPLACE, perturb=0.2, seed=3, qdeg=6)
    for c in [2, 19]:
        M, I, vol = exact.tet_exact(m.coords[m.cell_vert[c]], 3)
        np.testing.assert_allclose(pb.element_matrix(c), M, rtol=1e-11, atol=1e-15 * abs(M).max())
        K = np.einsum("abjj->ab", I)
        np.testing.assert_allclose(pl.element_matrix(c), K, rtol=1e-10, atol=1e-13 * abs(K).max())


@pytest.mark.parametrize("p", [3, 4, 6])
def test_tet_pk_conservation_and_null_spaces(p):
    nx = 2
    pb_m, m, nodes = tet_problem(nx, p, oracle.MASS, perturb=0.15, seed=5)
    pb_l, _, _ = tet_problem(nx, p, oracle.LAPLACE, perturb=0.15, seed=5)
    one = np.ones(pb_m.ndof)
    assert abs(pb_m.apply(one).sum() - 1.0) < 1e-13
    assert np.abs(pb_l.apply(one)).max() < 1e-12
    lin = 0.2 + nodes @ np.array([1.0, -0.7, 0.4])
    y = pb_l.apply(lin)
    inside = np.all((nodes > 1e-12) & (nodes < 1 - 1e-12), axis=1)
    assert inside.any() and np.abs(y[inside]).max() < 1e-12
    assert np.abs(y[~inside]).max() > 1e-4


@pytest.mark.parametrize("p", [3, 4])
def test_tet_pk_elasticity_rigid_modes_and_hyper_rotation(p):
    pb, m, nodes = tet_problem(2, p, oracle.ELASTICITY, perturb=0.15, seed=6, ncomp=3, lam=1.0, mu=1.0)
    for t in np.eye(3):
        assert np.abs(pb.apply(np.tile(t, (pb.nnode, 1)).ravel())).max() < 1e-13
    for w in np.eye(3):
        assert np.abs(pb.apply(np.cross(w, nodes).ravel())).max() < 1e-12
    ph, _, _ = tet_problem(2, p, oracle.HYPER_RES, perturb=0.15, seed=6, ncomp=3, law=oracle.NEOHOOKE, qdeg=2 * p)
    R = _rotation(0.5, [1, 1, -2])
    assert np.abs(ph.apply((nodes @ R.T - nodes).ravel())).max() < 1e-12


@pytest.mark.parametrize("which", ["tet-P2-elasticity", "quad-Q2-helmholtz", "tri-P3-laplace"])
def test_element_matrix_assembly_equals_unit_vector_matrix(which):
    """The assembled element matrices and the action on every unit vector give the same global matrix (the
    faster assembly stands in for dense() in the larger GPU tests)."""
    from tests.problems import assembled_dense, oracle_problem, quad_case, tet_case, tri_case

    case, kind = {"tet-P2-elasticity": (tet_case(1, 2, ncomp=3, perturb=0.1, seed=3), "elasticity"),
                  "quad-Q2-helmholtz": (quad_case(2, 2), "helmholtz"),
                  "tri-P3-laplace": (tri_case(2, 3), "laplace")}[which]
    pb = oracle_problem(case, kind)
    A1, A2 = pb.dense(), assembled_dense(pb, case)
    assert np.abs(A1 - A2).max() <= 1e-14 * np.abs(A1).max()
