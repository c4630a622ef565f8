"""Pins of the oracle's fully symmetric simplex rules (Table 2's 1/4/14/24 tet and 1/3/6/12 triangle points) to
facts outside the oracle: Table 2's point counts, exact integrals of random polynomials computed by sympy, the
closed-form 4- and 3-point rules, the symmetry group, and agreement of whole operator actions with the collapsed
rule wherever both rules are exact."""
import itertools
import math
import os

import numpy as np
import pytest

import fe_inputs as fi
import oracle
from oracle import symmetric
from tests.problems import tri_case, tet_case

HERE = os.path.dirname(os.path.abspath(__file__))
DEGREES = [(2, d) for d in range(0, 7)] + [(3, d) for d in range(0, 7)]


def table2_rows():
    return [l.split() for l in open(os.path.join(HERE, "golden", "table2_simplex_points.txt")) if l[0] != "#"]


@pytest.mark.parametrize("row", table2_rows(), ids=lambda r: "-".join(r))
def test_point_counts_match_table2(row):
    cell, _, _, degree, q = row
    dim, degree, q = (3 if cell == "tet" else 2), int(degree), int(q)
    if degree <= 6:
        pts, w = symmetric.rule(dim, degree)
        assert len(w) == q
    else:
        m = (degree + 2) // 2
        assert m ** dim == q
        pts, w = (oracle.tet_rule if dim == 3 else oracle.tri_rule)(degree)
        assert len(w) == q


def sympy_integral(dim, coef_exps):
    """Exact integral over the reference simplex of sum c x^a y^b (z^c) by sympy, as a float."""
    sp = pytest.importorskip("sympy")
    xs = sp.symbols("x0:%d" % dim)
    f = sum(sp.Rational(int(c)) * sp.prod([v ** int(e) for v, e in zip(xs, ex)]) for c, ex in coef_exps)
    if dim == 2:
        val = sp.integrate(f, (xs[1], 0, 1 - xs[0]), (xs[0], 0, 1))
    else:
        val = sp.integrate(f, (xs[2], 0, 1 - xs[0] - xs[1]), (xs[1], 0, 1 - xs[0]), (xs[0], 0, 1))
    return float(val)


@pytest.mark.parametrize("dim, degree", [(2, 2), (2, 3), (2, 4), (2, 5), (2, 6), (3, 2), (3, 3), (3, 4), (3, 5),
                                         (3, 6)])
def test_exact_for_random_polynomials_by_sympy(dim, degree):
    pts, w = symmetric.rule(dim, degree)
    rng = np.random.default_rng(100 * dim + degree)
    exps = [e for e in itertools.product(range(degree + 1), repeat=dim) if sum(e) <= degree]
    for trial in range(3):
        terms = [(int(rng.integers(-9, 10)), e) for e in exps]
        q = sum(c * (w * np.prod(pts ** np.array(e), axis=1)).sum() for c, e in terms)
        assert q == pytest.approx(sympy_integral(dim, terms), rel=1e-13, abs=1e-15)
    # one degree more than the rule's design degree is not integrated exactly: the rule is not over-provisioned
    design = symmetric.design_degree(dim, degree)
    top = [e for e in itertools.product(range(design + 2), repeat=dim) if sum(e) == design + 1]
    errs = [abs((w * np.prod(pts ** np.array(e), axis=1)).sum() - sympy_integral(dim, [(1, e)])) for e in top]
    assert max(errs) > 1e-8


def test_closed_form_low_order_rules():
    # tet, degree 2: the orbit (a, a, a, 1 - 3a), equal weights 1/24; the mean of l_1^2 over the tet is 1/10, so
    # (3a^2 + (1 - 3a)^2) / 4 = 1/10, whose root inside the tet is a = (5 - sqrt 5) / 20
    pts, w = symmetric.rule(3, 2)
    a = (5 - math.sqrt(5)) / 20
    bary = np.column_stack([1 - pts.sum(1), pts])
    assert np.allclose(np.sort(bary, axis=1), np.sort(np.array([[a, a, a, 1 - 3 * a]] * 4), axis=1), atol=1e-14)
    assert np.allclose(w, 1 / 24, atol=1e-16)
    # triangle, degree 2: (a, a, 1 - 2a) with (2a^2 + (1 - 2a)^2) / 3 = 1/6: a = 1/6 (or 1/2, on the edges)
    pts, w = symmetric.rule(2, 2)
    bary = np.column_stack([1 - pts.sum(1), pts])
    assert np.allclose(np.sort(bary, axis=1), np.sort(np.array([[1 / 6, 1 / 6, 2 / 3]] * 3), axis=1), atol=1e-14)
    assert np.allclose(w, 1 / 6, atol=1e-16)
    # degree <= 1: the centroid with the whole volume
    for dim in (2, 3):
        pts, w = symmetric.rule(dim, 1)
        assert np.allclose(pts, 1 / (dim + 1)) and w[0] == pytest.approx(1 / math.factorial(dim))


@pytest.mark.parametrize("dim, degree", [(2, 4), (2, 6), (3, 5), (3, 6)])
def test_symmetric_positive_interior(dim, degree):
    pts, w = symmetric.rule(dim, degree)
    bary = np.column_stack([1 - pts.sum(1), pts])
    assert w.min() > 0 and bary.min() > 0
    assert w.sum() == pytest.approx(1 / math.factorial(dim), rel=1e-14)
    key = {tuple(np.round(b, 10)): wi for b, wi in zip(bary, w)}
    for b, wi in zip(bary, w):  # every permutation of every point is a point of the rule, with the same weight
        for perm in itertools.permutations(range(dim + 1)):
            k = tuple(np.round(b[list(perm)], 10))
            assert k in key and key[k] == pytest.approx(wi, rel=1e-12)


@pytest.mark.parametrize("dim, degree, nsol", [(2, 4, 1), (2, 6, 2), (3, 5, 1), (3, 6, 1)])
def test_selection_is_unique(dim, degree, nsol):
    """Another seed finds the same admissible solutions; the rule taken is the one farthest from the boundary."""
    sols = symmetric.search(dim, degree, seed=99)
    assert len(sols) == nsol
    pts, w = symmetric.rule(dim, degree)
    bary = np.column_stack([1 - pts.sum(1), pts])
    best = sols[0][0]
    canon = lambda pts_: np.array(sorted(map(tuple, np.round(pts_, 8))))  # noqa: E731
    assert np.allclose(canon(bary), canon(best), atol=1e-8)
    if nsol == 2:
        assert sols[0][0].min() > sols[1][0].min() + 0.01


@pytest.mark.parametrize("cell, p, kind", [("tet", 1, "mass"), ("tet", 2, "helmholtz"), ("tet", 3, "mass"),
                                           ("tet", 3, "laplace"), ("tet", 4, "laplace"), ("tri", 1, "mass"),
                                           ("tri", 2, "helmholtz"), ("tri", 3, "mass"), ("tri", 4, "laplace")])
def test_actions_agree_with_collapsed_rule_when_exact(cell, p, kind):
    """A polynomial integrand of degree d is integrated exactly by both rule families: the actions agree to
    rounding (a wrong weight, point or scaling in either rule would show)."""
    case = tet_case(2, p, perturb=0.1, seed=3) if cell == "tet" else tri_case(3, p, seed=3)
    deg = 2 * p if kind in ("mass", "helmholtz") else 2 * (p - 1)
    x = fi.uniform_vector(case["nnode"], seed=5)
    ys = []
    for rule in ("collapsed", "symmetric"):
        pb = oracle.Problem(case["cell_type"], case["coords"], case["cell_vert"], p, case["cell_node"],
                            case["nnode"], {"mass": oracle.MASS, "laplace": oracle.LAPLACE,
                                            "helmholtz": oracle.HELMHOLTZ}[kind], qdeg=max(deg, 1), k2=0.7,
                            rule=rule)
        ys.append(pb.apply(x))
    assert np.linalg.norm(ys[0] - ys[1]) <= 1e-13 * np.linalg.norm(ys[0])


def test_nonpolynomial_integrand_depends_on_the_rule():
    """The neo-Hookean residual is not a polynomial: the 14-point and 27-point rules of degree 4/5 give close but
    different actions, and both approach a rule of high degree."""
    case = tet_case(2, 2, ncomp=3, perturb=0.1, seed=4)
    u = fi.sinusoid_displacement(case["nodes"], seed=6).ravel()
    ys = {}
    for name, qdeg, rule in [("sym", 4, "symmetric"), ("col", 4, "collapsed"), ("fine", 16, "collapsed")]:
        pb = oracle.Problem(case["cell_type"], case["coords"], case["cell_vert"], 2, case["cell_node"],
                            case["nnode"], oracle.HYPER_RES, ncomp=3, qdeg=qdeg, law=oracle.NEOHOOKE, rule=rule)
        ys[name] = pb.apply(u)
    n = np.linalg.norm(ys["fine"])
    assert np.linalg.norm(ys["sym"] - ys["col"]) > 1e-12 * n
    assert np.linalg.norm(ys["sym"] - ys["fine"]) < 1e-3 * n and np.linalg.norm(ys["col"] - ys["fine"]) < 1e-3 * n
