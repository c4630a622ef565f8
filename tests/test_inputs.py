"""The seeded input generators shared by the oracle and the GPU path (fe_inputs): SplitMix64 against its published
test vector, counter-based slicing, and meshes, maps and fields with the properties the readings ask for (boundary
kept, perturbation bounded, positive orientation, unit volume, conforming node counts)."""
import itertools

import numpy as np
import pytest

import fe_inputs as fi
from fe_inputs import rng


def test_splitmix64_published_vector():
    # SplitMix64 (Steele, Lea and Flood 2014) from state 0: outputs mix(k * GAMMA), k = 1, 2, 3
    with np.errstate(over="ignore"):
        z = rng._mix(np.arange(1, 4, dtype=np.uint64) * rng.GAMMA)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_counter_based_and_distinct():
    full = rng.splitmix64(7, 3, 20)
    assert np.array_equal(full[5:12], rng.splitmix64(7, 3, 7, start=5))
    assert not np.array_equal(full, rng.splitmix64(7, 4, 20))
    assert not np.array_equal(full, rng.splitmix64(8, 3, 20))
    u = rng.uniform(1, 2, 100000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    assert np.array_equal(fi.uniform_vector(50, seed=3), fi.uniform_vector(50, seed=3))
    r = rng.randint(5, 6, 10000, 2, 9)
    assert r.min() == 2 and r.max() == 9


def trilinear_det_at_corners(X):
    """det J at the 8 corners of each hex [c][8][3] (local vertex a + 2b + 4c at corner (a, b, c))."""
    out = []
    for a, b, c in itertools.product((0, 1), repeat=3):
        v = a + 2 * b + 4 * c
        dx = X[:, v ^ 1] - X[:, v]
        dy = X[:, v ^ 2] - X[:, v]
        dz = X[:, v ^ 4] - X[:, v]
        sgn = (1 if a == 0 else -1) * (1 if b == 0 else -1) * (1 if c == 0 else -1)
        out.append(sgn * np.einsum("ci,ci->c", dx, np.cross(dy, dz)))
    return np.array(out)


@pytest.mark.parametrize("nx", [3, 6])
def test_hex_mesh_boundary_perturbation_orientation_volume(nx):
    m = fi.hex_box_mesh(nx, perturb=0.1, seed=1)
    h = 1.0 / nx
    grid = np.array([(i, j, k) for k in range(nx + 1) for j in range(nx + 1) for i in range(nx + 1)]) * h
    d = m.coords - grid
    on_boundary = np.any((grid < 1e-12) | (grid > 1 - 1e-12), axis=1)
    assert np.abs(d[on_boundary]).max() == 0.0
    assert np.abs(d).max() <= 0.1 * h + 1e-15 and np.abs(d[~on_boundary]).max() > 0.05 * h
    X = m.coords[m.cell_vert]
    assert trilinear_det_at_corners(X).min() > 0
    # volume: det J of a trilinear map has degree <= 2 in each direction, so 2 Gauss points per direction are exact
    g = 0.5 + np.array([-1, 1]) / (2 * np.sqrt(3))
    vol = 0.0
    for xi, eta, zeta in itertools.product(g, g, g):
        f = np.array([[1 - xi, xi], [1 - eta, eta], [1 - zeta, zeta]])
        df = np.array([-1.0, 1.0])
        J = np.zeros((X.shape[0], 3, 3))
        for v in range(8):
            a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
            dN = np.array([df[a] * f[1, b] * f[2, c], f[0, a] * df[b] * f[2, c], f[0, a] * f[1, b] * df[c]])
            J += X[:, v, :, None] * dN[None, None, :]
        vol += np.linalg.det(J).sum() / 8
    assert abs(vol - 1.0) < 1e-13


def test_kuhn_tets_orientation_volume_and_valence():
    m = fi.kuhn_tet_mesh(4)
    X = m.coords[m.cell_vert]
    det = np.einsum("ci,ci->c", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))
    assert det.min() > 0 and abs(det.sum() / 6 - 1.0) < 1e-13
    valence = np.bincount(m.cell_vert.ravel(), minlength=m.coords.shape[0])
    interior = np.all((m.coords > 1e-12) & (m.coords < 1 - 1e-12), axis=1)
    assert np.all(valence[interior] == 24)  # Kuhn/Freudenthal: every interior vertex is in 24 tets
    mp = fi.kuhn_tet_mesh(4, perturb=0.1, seed=2)
    Xp = mp.coords[mp.cell_vert]
    detp = np.einsum("ci,ci->c", Xp[:, 1] - Xp[:, 0], np.cross(Xp[:, 2] - Xp[:, 0], Xp[:, 3] - Xp[:, 0]))
    assert detp.min() > 0 and abs(detp.sum() / 6 - 1.0) < 1e-13


def test_planar_meshes_orientation_and_area():
    t = fi.tri_mesh(5, perturb=0.15, seed=2)
    X = t.coords[t.cell_vert]
    a = 0.5 * ((X[:, 1, 0] - X[:, 0, 0]) * (X[:, 2, 1] - X[:, 0, 1]) - (X[:, 1, 1] - X[:, 0, 1]) * (X[:, 2, 0] - X[:, 0, 0]))
    assert a.min() > 0 and abs(a.sum() - 1.0) < 1e-14
    q = fi.quad_mesh(5, perturb=0.1, seed=1)
    Y = q.coords[q.cell_vert]  # local vertex v at corner (v & 1, v >> 1 & 1): 0, 1, 3, 2 is the counter-clockwise loop
    loop = Y[:, [0, 1, 3, 2], :2]
    area = 0.5 * np.sum(loop[:, :, 0] * np.roll(loop[:, :, 1], -1, axis=1) - np.roll(loop[:, :, 0], -1, axis=1) * loop[:, :, 1], axis=1)
    assert area.min() > 0 and abs(area.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 4])
def test_conforming_node_counts(p):
    nx = 3
    cn, nnode = fi.hex_node_map(nx, p)
    assert nnode == (nx * p + 1) ** 3 and np.array_equal(np.unique(cn), np.arange(nnode))
    cq, nq = fi.quad_node_map(nx, p)
    assert nq == (nx * p + 1) ** 2 and np.array_equal(np.unique(cq), np.arange(nq))
    t = fi.tri_mesh(nx)
    ct, nt, _ = fi.tri_node_map(t.cell_vert, t.coords.shape[0], p)
    assert nt == (nx * p + 1) ** 2 and np.array_equal(np.unique(ct), np.arange(nt))
    k = fi.kuhn_tet_mesh(nx)
    ck, nk, _ = fi.pk_node_map(k.cell_vert, k.coords.shape[0], p)
    assert nk == (nx * p + 1) ** 3 and np.array_equal(np.unique(ck), np.arange(nk))


def test_fields_bounds_and_determinism():
    pts = fi.kuhn_tet_mesh(3).coords
    u = fi.sinusoid_displacement(pts, seed=2)
    assert u.shape == (pts.shape[0], 3) and np.abs(u).max() <= 0.05 + 1e-15
    assert np.array_equal(u, fi.sinusoid_displacement(pts, seed=2))
    assert not np.array_equal(u, fi.sinusoid_displacement(pts, seed=3))
    g = fi.grf_lattice(9, seed=4)
    assert np.array_equal(g, fi.grf_lattice(9, seed=4)) and np.isfinite(g).all() and g.std() > 0
