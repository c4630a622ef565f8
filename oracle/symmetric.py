"""Fully symmetric quadrature rules on the reference triangle and tetrahedron (TEST INFRASTRUCTURE ONLY: used by
the oracle's `Problem(rule="symmetric")`, the tests and the benchmark's CPU leg, never by the library).

Table 2 (Section 4) integrates on simplices with 1, 4, 14 and 24 points (tetrahedra) and 1, 3, 6 and 12 points
(triangles) up to degree 6, and with collapsed product rules (m^3 and m^2 points) above.  The paper does not print
the points.  A fully symmetric rule is a union of orbits of the permutations of the barycentric coordinates,
with one weight per orbit; it is exact to degree d when it integrates every monomial of degree <= d exactly:

    (1/|T|) * integral over T of l_1^a1 ... l_n^an = a1! ... an! n! / (a1 + ... + an + n)!     (n = dim)

Orbit structures (orbit sizes sum to Table 2's counts):

    tet  d <= 1: centroid (1);  d = 2: S31 (4);  d <= 5: S31 + S31 + S22 (14);  d = 6: 3 x S31 + S211 (24)
    tri  d <= 1: centroid (1);  d = 2: S21 (3);  d <= 4: S21 + S21 (6);         d <= 6: 2 x S21 + S111 (12)

with S31 = (a, a, a, 1 - 3a), S22 = (a, a, 1/2 - a, 1/2 - a), S211 = (a, a, b, 1 - 2a - b), S21 = (a, a, 1 - 2a),
S111 = (a, b, 1 - a - b) and all their distinct permutations.  The moment equations are solved in the least
squares sense by variable projection: for given orbit positions the moment equations are linear in the weights,
which are solved for by linear least squares, and Levenberg-Marquardt (scipy) moves the positions from seeded
random starts inside the simplex to a zero of the remaining residual; the rule taken is then polished by
Gauss-Newton in extended precision (np.longdouble).  A solution is admissible when every
weight is positive and every point is strictly inside the simplex.  The rule taken is the admissible one whose
smallest barycentric coordinate is largest (its points are farthest from the boundary).  The only structures
with more than one admissible solution are the 12-point triangle rule, which has two, and the 3-point triangle
rule, whose second solution (the edge midpoints) lies on the boundary.
"""
import itertools
import math

import numpy as np

# orbit kind -> class pattern over the barycentric slots, number of free parameters
_PATTERN = {3: {"S31": (0, 0, 0, 1), "S22": (0, 0, 1, 1), "S211": (0, 0, 1, 2)},
            2: {"S21": (0, 0, 1), "S111": (0, 1, 2)}}
_NPARAM = {"S31": 1, "S22": 1, "S211": 2, "S21": 1, "S111": 2}
CENTROID = "centroid"


def structure(dim, degree):
    """Orbits of the symmetric rule of exactness `degree` (None above degree 6)."""
    if degree <= 1:
        return [CENTROID]
    if dim == 3:
        return {2: ["S31"], 3: ["S31", "S31", "S22"], 4: ["S31", "S31", "S22"], 5: ["S31", "S31", "S22"],
                6: ["S31", "S31", "S31", "S211"]}.get(degree)
    return {2: ["S21"], 3: ["S21", "S21"], 4: ["S21", "S21"], 5: ["S21", "S21", "S111"],
            6: ["S21", "S21", "S111"]}.get(degree)


def design_degree(dim, degree):
    """The degree a rule is solved for: Table 2's rules have exactness 1, 2, 5, 6 (tet) and 1, 2, 4, 6 (triangle),
    and a request of a lower degree takes the next rule (the moment equations of, say, degree 4 alone would leave a
    family of 14-point solutions)."""
    if degree <= 2:
        return max(degree, 1)
    if dim == 3:
        return 5 if degree <= 5 else 6
    return 4 if degree <= 4 else 6


def orbit(dim, kind, prm):
    """The distinct points (barycentric, [k][dim+1]) of one orbit."""
    if kind == CENTROID:
        return np.full((1, dim + 1), 1.0 / (dim + 1))
    if kind == "S31":
        cls = [prm[0], 1 - 3 * prm[0]]
    elif kind == "S22":
        cls = [prm[0], 0.5 - prm[0]]
    elif kind == "S211":
        cls = [prm[0], prm[1], 1 - 2 * prm[0] - prm[1]]
    elif kind == "S21":
        cls = [prm[0], 1 - 2 * prm[0]]
    else:  # S111
        cls = [prm[0], prm[1], 1 - prm[0] - prm[1]]
    pat = _PATTERN[dim][kind]
    keys = sorted({tuple(pat[j] for j in perm) for perm in itertools.permutations(range(dim + 1))})
    return np.array([[cls[c] for c in key] for key in keys])


def orbit_points(dim, struct, x):
    """Barycentric points of every orbit from the positions x (the orbits' parameters, in order), and the orbit
    index of each point."""
    pts, owner, i = [], [], 0
    for k, kind in enumerate(struct):
        n = 0 if kind == CENTROID else _NPARAM[kind]
        o = orbit(dim, kind, x[i:i + n])
        i += n
        pts.append(o)
        owner.extend([k] * len(o))
    return np.vstack(pts), np.array(owner)


def monomial_moments(dim, degree):
    """Exponents (in the first dim barycentric coordinates) of every monomial of degree <= degree, and the mean
    of each over the simplex (the closed form above)."""
    exps = np.array([e for e in itertools.product(range(degree + 1), repeat=dim) if sum(e) <= degree])
    mean = np.array([math.prod(math.factorial(k) for k in e) * math.factorial(dim) / math.factorial(sum(e) + dim)
                     for e in exps])
    return exps, mean


class MomentSystem:
    """The moment equations of one orbit structure, with the orbits' point patterns laid out once."""

    def __init__(self, dim, degree):
        self.dim, self.struct = dim, structure(dim, degree)
        self.exps, self.mean = monomial_moments(dim, degree)
        probe = np.arange(1, 1 + sum(_NPARAM.get(k, 0) for k in self.struct)) * 0.01
        bary, self.owner = orbit_points(dim, self.struct, probe)
        self.npts = len(self.owner)
        # each point coordinate as an affine function of the parameters: bary = const + lin @ x
        self.const = orbit_points(dim, self.struct, np.zeros_like(probe))[0]
        self.lin = np.stack([orbit_points(dim, self.struct, np.eye(len(probe))[j])[0] - self.const
                             for j in range(len(probe))], axis=-1)

    def points(self, x):
        return self.const + self.lin @ x

    def weights(self, x):
        """Least-squares orbit weights for the positions x, the point weights and the moment residual."""
        bary = self.points(x)
        vals = np.prod(bary[:, None, :self.dim] ** self.exps[None, :, :], axis=2)  # [point][monomial]
        per_orbit = np.zeros((len(self.struct), len(self.mean)))
        np.add.at(per_orbit, self.owner, vals)  # the rule's sum of each monomial over each orbit
        wo = np.linalg.lstsq(per_orbit.T, self.mean, rcond=None)[0]
        return wo, wo[self.owner], wo @ per_orbit - self.mean

    def residual(self, x):
        return self.weights(x)[2]

    def polish(self, x, iters=6):
        """Gauss-Newton on weights and positions together in extended precision (np.longdouble), from a double
        solution: the rule to well below double rounding, whatever the conditioning of the moment equations.
        Returns orbit weights and positions."""
        ld = np.longdouble
        wo = self.weights(x)[0]
        u = np.concatenate([wo, x]).astype(ld)
        norb, const, lin = len(self.struct), self.const.astype(ld), self.lin.astype(ld)
        exps, mean = self.exps, np.array([ld(m) for m in self.mean])
        for _ in range(iters):
            w, xs = u[:norb], u[norb:]
            bary = const + lin @ xs
            lam = bary[:, :self.dim]
            powers = [[lam[:, i] ** int(e) for e in range(exps.max() + 1)] for i in range(self.dim)]
            vals = np.ones((self.npts, len(mean)), dtype=ld)
            for q, ex in enumerate(exps):
                for i in range(self.dim):
                    vals[:, q] *= powers[i][ex[i]]
            wp = w[self.owner]
            r = wp @ vals - mean
            J = np.zeros((len(mean), len(u)), dtype=ld)
            for k in range(norb):
                J[:, k] = vals[self.owner == k].sum(axis=0)
            for q, ex in enumerate(exps):
                dm = np.zeros((self.npts, self.dim), dtype=ld)  # d(monomial)/d(lambda_i)
                for i in range(self.dim):
                    if ex[i] == 0:
                        continue
                    d = ld(int(ex[i])) * powers[i][ex[i] - 1]
                    for k in range(self.dim):
                        if k != i:
                            d = d * powers[k][ex[k]]
                    dm[:, i] = d
                J[q, norb:] = np.einsum("p,pi,pij->j", wp, dm, lin[:, :self.dim, :])
            u = u + _solve_ld(J.T @ J, -(J.T @ r))
        return u[:norb], u[norb:]


def _solve_ld(A, b):
    """Gaussian elimination with partial pivoting in the arrays' precision (LAPACK has no long double)."""
    A, b = A.copy(), b.copy()
    n = len(b)
    for c in range(n):
        piv = c + int(np.argmax(np.abs(A[c:, c])))
        A[[c, piv]], b[[c, piv]] = A[[piv, c]], b[[piv, c]]
        for r in range(c + 1, n):
            f = A[r, c] / A[c, c]
            A[r, c:] -= f * A[c, c:]
            b[r] -= f * b[c]
    x = np.zeros_like(b)
    for r in range(n - 1, -1, -1):
        x[r] = (b[r] - A[r, r + 1:] @ x[r + 1:]) / A[r, r]
    return x


def random_start(rng, struct):
    """Orbit positions drawn uniformly from the parameter ranges that keep the orbit inside the simplex."""
    x = []
    for kind in struct:
        if kind == "S31":
            x.append(rng.uniform(0, 1 / 3))
        elif kind == "S22":
            x.append(rng.uniform(0, 1 / 4))
        elif kind == "S21":
            x.append(rng.uniform(0, 1 / 2))
        elif kind == "S211":
            a = rng.uniform(0, 1 / 2)
            x.extend([a, rng.uniform(0, 1 - 2 * a)])
        elif kind == "S111":
            a = rng.uniform(0, 1)
            x.extend([a, rng.uniform(0, 1 - a)])
    return np.array(x)


def admissible(bary, w, margin=1e-9):
    return bool(w.min() > 0 and bary.min() > margin)


def search(dim, degree, starts=None, seed=0, tol=1e-13, keep_x=False):
    """Every distinct admissible solution found from `starts` seeded random starts, with the number of starts
    that reached it: a list of (barycentric points, weights, hits), best first by the selection rule."""
    from scipy.optimize import least_squares

    struct = structure(dim, degree)
    if struct is None:
        raise ValueError("no symmetric rule of degree %d on the %d-simplex" % (degree, dim))
    if struct == [CENTROID]:
        one = (np.full((1, dim + 1), 1.0 / (dim + 1)), np.ones(1), starts)
        return [(None,) + one + (None,)] if keep_x else [one]
    system = MomentSystem(dim, degree)
    if starts is None:  # about 1 start in 40 reaches the 24-point rule, 1 in 4 or more the others
        starts = 400 if len(system.owner) == 24 else 200
    rng = np.random.default_rng(seed)
    found = []
    for _ in range(starts):
        r = least_squares(system.residual, random_start(rng, struct), method="lm", xtol=1e-15, ftol=1e-15,
                          gtol=1e-15, max_nfev=100)  # converging starts take at most ~70 evaluations
        _, w, res = system.weights(r.x)
        if np.abs(res).max() > tol:
            continue
        bary = system.points(r.x)
        if not admissible(bary, w):
            continue
        key = np.array(sorted(map(tuple, np.round(bary, 8))))
        for item in found:
            if item[0].shape == key.shape and np.allclose(item[0], key, atol=1e-7):
                item[3] += 1
                break
        else:
            found.append([key, bary, w, 1, r.x])
    found.sort(key=lambda it: -it[1].min())
    return [(bary, w, hits) for _, bary, w, hits, _ in found] if not keep_x else found


_CACHE = {}


def rule(dim, degree):
    """The symmetric rule of exactness `degree` on the reference simplex (vertices 0, e_1, ..., e_dim): reference
    points [nq][dim] (the barycentric coordinates of vertices 1..dim) and weights summing to 1/dim!."""
    degree = design_degree(dim, degree)
    key = (dim, degree)
    if key not in _CACHE:
        sols = search(dim, degree, keep_x=True)
        if not sols:
            raise RuntimeError("no admissible symmetric rule of degree %d found" % degree)
        bary, w, x = sols[0][1], sols[0][2], sols[0][4]
        if x is not None and len(x):
            system = MomentSystem(dim, degree)
            wo, xs = system.polish(x)
            bary = (system.const.astype(np.longdouble) + system.lin.astype(np.longdouble) @ xs).astype(float)
            w = wo[system.owner].astype(float)
        _CACHE[key] = (np.ascontiguousarray(bary[:, 1:]), w / math.factorial(dim))
    pts, w = _CACHE[key]
    return pts.copy(), w.copy()
