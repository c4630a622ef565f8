"""Exact reference computations for the oracle pins, independent of the oracle.

Everything here uses either closed forms or numpy's polynomial routines; none
of it calls the oracle's quadrature, basis or geometry code.
"""
import math

import numpy as np
from numpy.polynomial import Legendre
from numpy.polynomial import legendre as L


def gll_nodes_np(n):
    """GLL nodes on [0,1] from numpy: endpoints and the roots of P_{n-1}'."""
    if n == 2:
        return np.array([0.0, 1.0])
    c = np.zeros(n)
    c[-1] = 1.0
    r = np.sort(L.legroots(L.legder(c)).real)
    return np.concatenate([[0.0], 0.5 * (1.0 + r), [1.0]])


def lagrange_polys(nodes):
    """1D Lagrange basis on ``nodes`` as numpy Legendre series on the domain [0,1]."""
    out = []
    for i, si in enumerate(nodes):
        others = [s for j, s in enumerate(nodes) if j != i]
        p = Legendre.fromroots(others, domain=[0.0, 1.0])
        out.append(p / p(si))
    return out


def int01(p):
    q = p.integ()
    return q(1.0) - q(0.0)


def matrices_1d(nodes):
    """Exact 1D integrals on [0,1]: M_ij = int l_i l_j, K_ij = int l_i' l_j', C_ij = int l_i' l_j."""
    ls = lagrange_polys(nodes)
    ds = [l.deriv() for l in ls]
    n = len(ls)
    M = np.array([[int01(ls[i] * ls[j]) for j in range(n)] for i in range(n)])
    K = np.array([[int01(ds[i] * ds[j]) for j in range(n)] for i in range(n)])
    C = np.array([[int01(ds[i] * ls[j]) for j in range(n)] for i in range(n)])
    return M, K, C


def affine_hex_matrices(p, A, kind, k2=1.0):
    """Exact element matrix of Q_p (GLL nodes) on the affine image x = A xi + b of [0,1]^3.

    Local index i + n j + n^2 k; the reference integrals factor into 1D ones.
    """
    nodes = gll_nodes_np(p + 1)
    M, K, C = matrices_1d(nodes)
    detA = abs(np.linalg.det(A))
    Ainv = np.linalg.inv(A)
    G = Ainv @ Ainv.T  # grad phi . grad psi = grad_ref phi^T G grad_ref psi
    one = [M, M, M]

    def kron3(mats):
        # index i + n j + n^2 k -> kron(z, y, x)
        return np.kron(mats[2], np.kron(mats[1], mats[0]))

    mass = detA * kron3(one)
    if kind == "mass":
        return mass
    stiff = np.zeros_like(mass)
    for a in range(3):
        for b in range(3):
            mats = []
            for d in range(3):
                if d == a and d == b:
                    mats.append(K)
                elif d == a:       # derivative on test function in direction a
                    mats.append(C)  # C_ij = int l_i' l_j : test i differentiated
                elif d == b:
                    mats.append(C.T)
                else:
                    mats.append(M)
            stiff += G[a, b] * kron3(mats)
    stiff *= detA
    if kind == "laplace":
        return stiff
    return stiff + k2 * mass


# ---- exact integrals of barycentric polynomials on a tetrahedron ----

def bary_integral(exps, vol):
    """int_K lambda0^a lambda1^b lambda2^c lambda3^d = 3! vol a! b! c! d! / (a+b+c+d+3)!."""
    num = math.factorial(3) * vol
    for e in exps:
        num *= math.factorial(e)
    return num / math.factorial(sum(exps) + 3)


def _pmul(p, q):
    r = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            r[e] = r.get(e, 0.0) + ca * cb
    return r


def _pdiff(p, k):
    r = {}
    for e, c in p.items():
        if e[k] > 0:
            f = list(e)
            f[k] -= 1
            r[tuple(f)] = r.get(tuple(f), 0.0) + c * e[k]
    return r


def _unit(k):
    e = [0, 0, 0, 0]
    e[k] = 1
    return tuple(e)


P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def pk_basis_bary(p):
    """P_p Lagrange basis on the equispaced lattice (p >= 3) as polynomials in the barycentric coordinates, by the
    closed product form prod_s prod_{t < b_s} (p lambda_s - t) / (t + 1) (Silvester), in exact rational arithmetic.
    Node order: lattice points (i, j, l)/p, i fastest, then j, then l; b = (p - i - j - l, i, j, l)."""
    from fractions import Fraction

    basis = []
    for l in range(p + 1):
        for j in range(p + 1 - l):
            for i in range(p + 1 - l - j):
                b = (p - i - j - l, i, j, l)
                poly = {(0, 0, 0, 0): Fraction(1)}
                for s in range(4):
                    for tt in range(b[s]):
                        lin = {_unit(s): Fraction(p, tt + 1)}
                        if tt:
                            lin[(0, 0, 0, 0)] = Fraction(-tt, tt + 1)
                        poly = _pmul(poly, lin)
                basis.append({e: float(c) for e, c in poly.items() if c != 0})
    return basis


def p_basis_bary(p):
    """Lagrange basis as polynomials in the barycentric coordinates (P1/P2 closed forms, P3+ by pk_basis_bary)."""
    if p >= 3:
        return pk_basis_bary(p)
    if p == 1:
        return [{_unit(k): 1.0} for k in range(4)]
    basis = []
    for k in range(4):  # lambda_k (2 lambda_k - 1)
        e2 = [0, 0, 0, 0]
        e2[k] = 2
        basis.append({tuple(e2): 2.0, _unit(k): -1.0})
    for a, b in P2_EDGES:  # 4 lambda_a lambda_b
        e = [0, 0, 0, 0]
        e[a] += 1
        e[b] += 1
        basis.append({tuple(e): 4.0})
    return basis


def tet_exact(X, p):
    """Exact mass M_ab and gradient-product tensor I[a,b,j,l] = int d_j phi_a d_l phi_b on tet X [4][3]."""
    T = np.array([X[1] - X[0], X[2] - X[0], X[3] - X[0]]).T
    vol = abs(np.linalg.det(T)) / 6.0
    # barycentric gradients: lambda_{1..3} = T^{-1}(x - X0), lambda_0 = 1 - sum
    Ti = np.linalg.inv(T)
    gl = np.zeros((4, 3))
    gl[1:] = Ti
    gl[0] = -Ti.sum(axis=0)
    basis = p_basis_bary(p)
    n = len(basis)

    def integ(poly):
        return sum(c * bary_integral(e, vol) for e, c in poly.items())

    M = np.array([[integ(_pmul(basis[a], basis[b])) for b in range(n)] for a in range(n)])
    dB = [[_pdiff(basis[a], k) for k in range(4)] for a in range(n)]
    I = np.zeros((n, n, 3, 3))
    for a in range(n):
        for b in range(n):
            # int (sum_k dphi_a/dl_k grad l_k)_j (sum_m dphi_b/dl_m grad l_m)_l
            S = np.zeros((4, 4))
            for k in range(4):
                for m in range(4):
                    S[k, m] = integ(_pmul(dB[a][k], dB[b][m]))
            I[a, b] = gl.T @ S @ gl
    return M, I, vol
