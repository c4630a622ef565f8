"""FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under test never does, and
this package never imports the library: it is an independent restatement of
what the matrix-free operator action computes (arXiv 1903.08243, Section 2
and the Supplementary material), compiled from ``oracle.c`` with gcc.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")

TET, HEX, TRI, QUAD = 4, 8, 3, 40
MASS, LAPLACE, HELMHOLTZ, ELASTICITY, HYPER_RES, HYPER_JAC = range(6)
SVK, NEOHOOKE = 0, 1


def build(force=False):
    """Compile oracle.c into liboracle.so (plain C11, -O2, no vector flags)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("cell_type", ctypes.c_int32),
        ("degree", ctypes.c_int32),
        ("ncomp", ctypes.c_int32),
        ("kind", ctypes.c_int32),
        ("law", ctypes.c_int32),
        ("qdeg", ctypes.c_int32),
        ("equispaced", ctypes.c_int32),
        ("nq_rule", ctypes.c_int32),
        ("ncell", ctypes.c_int64),
        ("nvert", ctypes.c_int64),
        ("nnode", ctypes.c_int64),
        ("coords", ctypes.c_void_p),
        ("cell_vert", ctypes.c_void_p),
        ("cell_node", ctypes.c_void_p),
        ("k2", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("b", ctypes.c_double * 3),
        ("ucoef", ctypes.c_void_p),
        ("qpts", ctypes.c_void_p),
        ("qw", ctypes.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, i64 = ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int64
        _lib.orc_gauss_legendre.argtypes = [i, d, d]
        _lib.orc_gauss_jacobi.argtypes = [i, i, d, d]
        _lib.orc_gll_nodes.argtypes = [i, d]
        _lib.orc_tet_rule.argtypes = [i, d, d]
        _lib.orc_tet_basis.argtypes = [i, d, d, d]
        _lib.orc_hex_basis.argtypes = [i, i, d, d, d]
        _lib.orc_tri_rule.argtypes = [i, d, d]
        _lib.orc_tri_basis.argtypes = [i, d, d, d]
        _lib.orc_quad_basis.argtypes = [i, d, d, d]
        _lib.orc_apply.argtypes = [ctypes.POINTER(_Problem), d, d, ctypes.POINTER(ctypes.c_int64), i64]
        _lib.orc_energy.argtypes = [ctypes.POINTER(_Problem), d, d]
        _lib.orc_element_matrix.argtypes = [ctypes.POINTER(_Problem), i64, d]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc < 0:
        raise OracleError("%s failed with code %d" % (what, rc))
    return rc


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_legendre(n, _dp(x), _dp(w)), "gauss_legendre")
    return x, w


def gauss_jacobi(n, alpha):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_jacobi(n, alpha, _dp(x), _dp(w)), "gauss_jacobi")
    return x, w


def gll_nodes(n):
    x = np.zeros(n)
    _check(lib().orc_gll_nodes(n, _dp(x)), "gll_nodes")
    return x


def tet_rule(degree):
    m = (degree + 2) // 2
    pts, w = np.zeros((m ** 3, 3)), np.zeros(m ** 3)
    _check(lib().orc_tet_rule(degree, _dp(pts), _dp(w)), "tet_rule")
    return pts, w


def tet_basis(p, xi):
    n = (p + 1) * (p + 2) * (p + 3) // 6
    phi, dphi = np.zeros(n), np.zeros((n, 3))
    _check(lib().orc_tet_basis(p, _dp(np.ascontiguousarray(xi, dtype=np.float64)), _dp(phi), _dp(dphi)), "tet_basis")
    return phi, dphi


def hex_basis(p, xi, equispaced=False):
    n = (p + 1) ** 3
    phi, dphi = np.zeros(n), np.zeros((n, 3))
    _check(
        lib().orc_hex_basis(p, int(equispaced), _dp(np.ascontiguousarray(xi, dtype=np.float64)), _dp(phi), _dp(dphi)),
        "hex_basis",
    )
    return phi, dphi


def tri_rule(degree):
    m = (degree + 2) // 2
    pts, w = np.zeros((m * m, 2)), np.zeros(m * m)
    _check(lib().orc_tri_rule(degree, _dp(pts), _dp(w)), "tri_rule")
    return pts, w


def tri_basis(p, xi):
    n = (p + 1) * (p + 2) // 2
    phi, dphi = np.zeros(n), np.zeros((n, 2))
    _check(lib().orc_tri_basis(p, _dp(np.ascontiguousarray(xi, dtype=np.float64)), _dp(phi), _dp(dphi)), "tri_basis")
    return phi, dphi


def quad_basis(p, xi):
    n = (p + 1) ** 2
    phi, dphi = np.zeros(n), np.zeros((n, 2))
    _check(lib().orc_quad_basis(p, _dp(np.ascontiguousarray(xi, dtype=np.float64)), _dp(phi), _dp(dphi)), "quad_basis")
    return phi, dphi


class Problem:
    """A mesh, a space and a form, held as arrays the C oracle reads."""

    def __init__(self, cell_type, coords, cell_vert, degree, cell_node, nnode, kind, ncomp=1,
                 qdeg=None, k2=1.0, lam=1.0, mu=1.0, law=SVK, b=(0.0, 0.0, 0.0), ucoef=None,
                 equispaced=False, rule="collapsed"):
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.cell_vert = np.ascontiguousarray(cell_vert, dtype=np.int32)
        self.cell_node = np.ascontiguousarray(cell_node, dtype=np.int32)
        self.ucoef = None if ucoef is None else np.ascontiguousarray(ucoef, dtype=np.float64).ravel()
        if qdeg is None:
            qdeg = degree + 1 if cell_type in (HEX, QUAD) else 2 * degree
        s = _Problem()
        s.cell_type, s.degree, s.ncomp, s.kind, s.law, s.qdeg = cell_type, degree, ncomp, kind, law, qdeg
        s.equispaced = int(equispaced)
        s.ncell, s.nvert, s.nnode = self.cell_vert.shape[0], self.coords.shape[0], nnode
        s.coords = self.coords.ctypes.data
        s.cell_vert = self.cell_vert.ctypes.data
        s.cell_node = self.cell_node.ctypes.data
        s.k2, s.lam, s.mu = k2, lam, mu
        s.b[0], s.b[1], s.b[2] = b
        s.ucoef = None if self.ucoef is None else self.ucoef.ctypes.data
        if rule not in ("collapsed", "symmetric"):
            raise ValueError("rule must be 'collapsed' or 'symmetric'")
        if rule == "symmetric" and cell_type in (TET, TRI) and qdeg <= 6:
            # Table 2's fully symmetric rules up to degree 6 (the collapsed rule above)
            from oracle import symmetric
            pts, w = symmetric.rule(3 if cell_type == TET else 2, qdeg)
            self._qpts, self._qw = np.ascontiguousarray(pts), np.ascontiguousarray(w)
            s.nq_rule, s.qpts, s.qw = len(w), self._qpts.ctypes.data, self._qw.ctypes.data
        self._s = s
        self.ncomp = ncomp
        self.nnode = nnode
        self.ndof = nnode * ncomp

    def apply(self, x, cells=None):
        x = np.ascontiguousarray(x, dtype=np.float64).ravel()
        if x.size != self.ndof:
            raise ValueError("x has %d entries, expected %d" % (x.size, self.ndof))
        y = np.zeros(self.ndof)
        if cells is None:
            rc = lib().orc_apply(ctypes.byref(self._s), _dp(x), _dp(y), None, 0)
        else:
            c = np.ascontiguousarray(cells, dtype=np.int64)
            rc = lib().orc_apply(ctypes.byref(self._s), _dp(x), _dp(y),
                                 c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), c.size)
        _check(rc, "apply")
        return y

    def energy(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64).ravel()
        e = np.zeros(1)
        _check(lib().orc_energy(ctypes.byref(self._s), _dp(u), _dp(e)), "energy")
        return float(e[0])

    def element_matrix(self, cell):
        m = self.cell_node.shape[1] * self.ncomp
        A = np.zeros((m, m))
        _check(lib().orc_element_matrix(ctypes.byref(self._s), cell, _dp(A)), "element_matrix")
        return A

    def dense(self):
        """Global matrix by applying the operator to every unit vector (tiny meshes only)."""
        n = self.ndof
        if n > 4000:
            raise ValueError("dense() is for tiny meshes")
        A = np.zeros((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[:] = 0.0
            e[j] = 1.0
            A[:, j] = self.apply(e)
        return A
