"""The library's own cell -> node maps (host code, no GPU): conforming under any local vertex order, equal to the
input generators' maps up to a renumbering of the nodes, and giving the same operator (checked with the oracle)."""
import itertools

import numpy as np
import pytest

import fe_inputs as fi
import oracle
import paper_1903_08243_gb300 as mfa
from tests import exact
from tests.problems import hex_node_coords


def same_partition(a, b):
    """True if the two cell -> node maps differ only by a renumbering of the nodes."""
    fwd, bwd = {}, {}
    for x, y in zip(a.ravel().tolist(), b.ravel().tolist()):
        if fwd.setdefault(x, y) != y or bwd.setdefault(y, x) != x:
            return False
    return True


def cube_rotations():
    """The 24 rotations of the reference cube as permutations of its corners (corner v at bits of v)."""
    out = []
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product([0, 1], repeat=3):
            M = np.zeros((3, 3), int)
            for r in range(3):
                M[r, perm[r]] = -1 if flips[r] else 1
            if round(np.linalg.det(M)) != 1:
                continue
            corners = np.array([[(v >> d) & 1 for d in range(3)] for v in range(8)])
            img = (corners - 0.5) @ M.T + 0.5
            idx = [int(round(c[0] + 2 * c[1] + 4 * c[2])) for c in img]
            out.append(idx)
    return out


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_hex_map_equals_the_structured_map(p):
    nx = 3
    mesh = fi.hex_box_mesh(nx)
    cn_ref, nn_ref = fi.hex_node_map(nx, p)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_HEX8, p, mesh.cell_vert, mesh.nvert)
    assert nn == nn_ref and same_partition(cn, cn_ref)
    X = mfa.mfa_node_coords(mfa.MFA_CELL_HEX8, p, mesh.cell_vert, mesh.coords, cn, nn)
    Xr = hex_node_coords(mesh, cn_ref, p)
    np.testing.assert_allclose(X[cn], Xr[cn_ref], atol=1e-14)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_hex_map_is_conforming_under_rotated_local_orders(p):
    """Every cell's local vertex order rotated by a random rotation of the cube: the nodes each cell sees at its
    own GLL points must be the same global nodes (checked through their physical positions), and the operator
    must be the same up to that renumbering."""
    nx = 2
    mesh = fi.hex_box_mesh(nx, perturb=0.1, seed=4)
    rots = cube_rotations()
    assert len(rots) == 24
    rng = np.random.default_rng(p)
    cv = np.array([mesh.cell_vert[c][rots[rng.integers(24)]] for c in range(mesh.cell_vert.shape[0])],
                  dtype=np.int32)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_HEX8, p, cv, mesh.nvert)
    assert nn == (nx * p + 1) ** 3
    # positions seen from each cell agree for every shared node
    n = p + 1
    s = exact.gll_nodes_np(n)
    seen = {}
    for c in range(cv.shape[0]):
        X = mesh.coords[cv[c]]
        for k, j, i in itertools.product(range(n), repeat=3):
            xi = (s[i], s[j], s[k])
            w = np.array([np.prod([xi[d] if (v >> d) & 1 else 1 - xi[d] for d in range(3)]) for v in range(8)])
            pos = w @ X
            node = cn[c, i + n * (j + n * k)]
            if node in seen:
                np.testing.assert_allclose(seen[node], pos, atol=1e-13)
            else:
                seen[node] = pos
    assert len(seen) == nn
    # same operator as on the generator's map, up to the renumbering
    cn_ref, _ = fi.hex_node_map(nx, p)
    ref = oracle.Problem(oracle.HEX, mesh.coords, mesh.cell_vert, p, cn_ref, nn, oracle.LAPLACE, qdeg=p + 1)
    pb = oracle.Problem(oracle.HEX, mesh.coords, cv, p, cn, nn, oracle.LAPLACE, qdeg=p + 1)
    Xr = hex_node_coords(mesh, cn_ref, p)
    Xn = np.array([seen[v] for v in range(nn)])
    key = lambda X: np.round(X * 1e9).astype(np.int64).tolist()
    pos_ref = {tuple(k): i for i, k in enumerate(key(Xr))}
    perm = np.array([pos_ref[tuple(k)] for k in key(Xn)])  # new node -> reference node
    x_ref = fi.uniform_vector(nn, seed=5)
    np.testing.assert_allclose(pb.apply(x_ref[perm]), ref.apply(x_ref)[perm], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_tet_map_equals_the_generator_maps(p):
    mesh = fi.kuhn_tet_mesh(3)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_TET4, p, mesh.cell_vert, mesh.nvert)
    if p == 1:
        cn_ref, nn_ref = mesh.cell_vert, mesh.nvert
    elif p == 2:
        cn_ref, nn_ref, _ = fi.p2_node_map(mesh.cell_vert, mesh.nvert)
    else:
        cn_ref, nn_ref, _ = fi.pk_node_map(mesh.cell_vert, mesh.nvert, p)
    assert nn == nn_ref and same_partition(cn, cn_ref)
    assert np.array_equal(cn[:, :1], cn_ref[:, :1]) or p >= 3  # vertex nodes keep the vertex ids


def test_tet_map_conforming_under_permuted_local_orders():
    """Even permutations of each tet's local vertices (orientation kept): shared nodes at equal positions."""
    p = 4
    mesh = fi.kuhn_tet_mesh(2, perturb=0.1, seed=2)
    rng = np.random.default_rng(7)
    even = [q for q in itertools.permutations(range(4))
            if sum(1 for i in range(4) for j in range(i + 1, 4) if q[i] > q[j]) % 2 == 0]
    cv = np.array([c[list(even[rng.integers(len(even))])] for c in mesh.cell_vert], dtype=np.int32)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_TET4, p, cv, mesh.nvert)
    lat = fi.pk_lattice(p)
    seen = {}
    for c in range(cv.shape[0]):
        X = mesh.coords[cv[c]]
        for a in range(lat.shape[0]):
            pos = (lat[a] / p) @ X
            node = cn[c, a]
            if node in seen:
                np.testing.assert_allclose(seen[node], pos, atol=1e-13)
            else:
                seen[node] = pos
    assert len(seen) == nn == (2 * p + 1) ** 3


def test_map_builder_errors():
    cv = np.array([[0, 1, 2, 3]], dtype=np.int32)
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_build_cell_node(mfa.MFA_CELL_TET4, 7, cv, 4)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_build_cell_node(mfa.MFA_CELL_TET4, 2, cv, 3)  # vertex 3 outside [0, 3)
    assert e.value.code == mfa.MFA_ERR_RANGE


@pytest.mark.parametrize("p", [1, 2, 4])
def test_planar_maps_equal_the_generator_maps(p):
    q = fi.quad_mesh(4)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_QUAD4, p, q.cell_vert, q.nvert)
    cn_ref, nn_ref = fi.quad_node_map(4, p)
    assert nn == nn_ref and same_partition(cn, cn_ref)
    t = fi.tri_mesh(4)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_TRI3, p, t.cell_vert, t.nvert)
    cn_ref, nn_ref, _ = fi.tri_node_map(t.cell_vert, t.nvert, p)
    assert nn == nn_ref and same_partition(cn, cn_ref)


def test_quad_map_conforming_under_rotated_local_orders():
    p = 3
    q = fi.quad_mesh(3, perturb=0.1, seed=2)
    rots = [[0, 1, 2, 3], [1, 3, 0, 2], [3, 2, 1, 0], [2, 0, 3, 1]]  # the 4 rotations of the square's corners
    rng = np.random.default_rng(1)
    cv = np.array([c[rots[rng.integers(4)]] for c in q.cell_vert], dtype=np.int32)
    cn, nn = mfa.mfa_build_cell_node(mfa.MFA_CELL_QUAD4, p, cv, q.nvert)
    n = p + 1
    s = exact.gll_nodes_np(n)
    seen = {}
    for c in range(cv.shape[0]):
        X = q.coords[cv[c]]
        for j in range(n):
            for i in range(n):
                w = np.array([(s[i] if v & 1 else 1 - s[i]) * (s[j] if v & 2 else 1 - s[j]) for v in range(4)])
                pos = w @ X
                node = cn[c, i + n * j]
                if node in seen:
                    np.testing.assert_allclose(seen[node], pos, atol=1e-13)
                else:
                    seen[node] = pos
    assert len(seen) == nn == (3 * p + 1) ** 2
