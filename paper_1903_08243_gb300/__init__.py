"""Python binding of libmfa: matrix-free finite element operator action on GB300.

Argument marshalling only.  Every step of the operator action runs in the
CUDA kernels of ``libmfa.so`` behind the C ABI of ``include/mfa.h``; this
module converts numpy arrays and torch CUDA tensors into pointers and status
codes into exceptions.  There is no CPU fallback: if the library is missing
the import fails.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmfa.so")

# ---- constants mirrored from include/mfa.h
MFA_OK, MFA_ERR_ARG, MFA_ERR_RANGE, MFA_ERR_UNSUPPORTED, MFA_ERR_CUDA = 0, 1, 2, 3, 4
MFA_ERR_OOM, MFA_ERR_TIMEOUT, MFA_ERR_NOT_CONVERGED, MFA_ERR_BREAKDOWN, MFA_ERR_DOMAIN = 5, 6, 7, 8, 9
MFA_CELL_TRI3, MFA_CELL_TET4, MFA_CELL_HEX8, MFA_CELL_QUAD4 = 3, 4, 8, 40
MFA_FORM_MASS, MFA_FORM_LAPLACE, MFA_FORM_HELMHOLTZ = 0, 1, 2
MFA_FORM_ELASTICITY, MFA_FORM_HYPER_RES, MFA_FORM_HYPER_JAC = 3, 4, 5
MFA_LAW_SVK, MFA_LAW_NEOHOOKE = 0, 1
MFA_PREC_FP64, MFA_PREC_FP32, MFA_PREC_BF16 = 0, 1, 2
MFA_GEOM_STORED, MFA_GEOM_ONTHEFLY = 0, 1
MFA_RULE_AUTO, MFA_RULE_SYMMETRIC = 0, 1
MFA_SCATTER_AUTO, MFA_SCATTER_COLOUR, MFA_SCATTER_ATOMIC, MFA_SCATTER_WARP = 0, 1, 2, 3
MFA_PC_NONE, MFA_PC_JACOBI = 0, 1
MFA_PRECOND_MLP, MFA_PRECOND_LINEAR = 0, 1
(MFA_VARIANT_AUTO, MFA_VARIANT_POINT, MFA_VARIANT_EVEN_ODD, MFA_VARIANT_LINE, MFA_VARIANT_LINE_STAGED,
 MFA_VARIANT_CELL, MFA_VARIANT_CELL_WARP) = 0, 1, 2, 3, 4, 5, 6
VARIANT_NAMES = {1: "point", 2: "even-odd", 3: "line", 4: "line-staged", 5: "cell", 6: "cell-warp"}


class MfaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mfa status %d: %s" % (code, msg))
        self.code = code


class mfa_form_params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("law", ctypes.c_int32),
        ("qdeg", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("scatter", ctypes.c_int32),
        ("cells_per_block", ctypes.c_int32),
        ("k2", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("b", ctypes.c_double * 3),
        ("geometry", ctypes.c_int32),
        ("rule", ctypes.c_int32),
    ]


class mfa_form_info(ctypes.Structure):
    _fields_ = [
        ("ncell", ctypes.c_int64),
        ("ndof", ctypes.c_int64),
        ("nloc", ctypes.c_int32),
        ("nq", ctypes.c_int32),
        ("ncolours", ctypes.c_int32),
        ("scatter", ctypes.c_int32),
        ("flops", ctypes.c_double),
        ("bytes", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("flops_executed", ctypes.c_double),
    ]


class mfa_launch_config(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int32),
        ("cells_per_block", ctypes.c_int32),
        ("scatter", ctypes.c_int32),
        ("geometry", ctypes.c_int32),
        ("max_blocks", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("ms", ctypes.c_double),
    ]

    def as_dict(self):
        return {"variant": VARIANT_NAMES.get(self.variant, self.variant), "cells_per_block": self.cells_per_block,
                "scatter": {MFA_SCATTER_COLOUR: "colour", MFA_SCATTER_WARP: "warp"}.get(self.scatter, "atomic"),
                "geometry": "on-the-fly" if self.geometry == MFA_GEOM_ONTHEFLY else "stored",
                "max_blocks": self.max_blocks, "ms": self.ms}


_lib = None
_VP, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)
_SIGS = {
    "mfa_last_error": ([], ctypes.c_char_p),
    "mfa_version": ([], _I),
    "mfa_create": ([_PP, _I, _VP], _I),
    "mfa_set_stream": ([_VP, _VP], _I),
    "mfa_destroy": ([_VP], _I),
    "mfa_mesh_upload": ([_VP, _I, _I64, _I64, _VP, _VP, _PP], _I),
    "mfa_mesh_destroy": ([_VP], _I),
    "mfa_space_create": ([_VP, _VP, _I, _I, _VP, _I64, _PP], _I),
    "mfa_space_get_cell_node": ([_VP, _VP], _I),
    "mfa_build_cell_node": ([_I, _I, _I64, _VP, _I64, _VP, ctypes.POINTER(_I64)], _I),
    "mfa_node_coords": ([_I, _I, _I64, _VP, _VP, _VP, _I64, _VP], _I),
    "mfa_simplex_rule": ([_I, _I, _I, _VP, _VP, ctypes.POINTER(_I)], _I),
    "mfa_space_ndof": ([_VP, ctypes.POINTER(_I64)], _I),
    "mfa_space_destroy": ([_VP], _I),
    "mfa_form_create": ([_VP, _VP, ctypes.POINTER(mfa_form_params), _PP], _I),
    "mfa_form_set_coefficient": ([_VP, _VP], _I),
    "mfa_form_get_info": ([_VP, ctypes.POINTER(mfa_form_info)], _I),
    "mfa_form_destroy": ([_VP], _I),
    "mfa_form_set_dirichlet": ([_VP, _VP, _I64], _I),
    "mfa_form_list_configs": ([_VP, _VP, _I, ctypes.POINTER(_I)], _I),
    "mfa_form_get_config": ([_VP, ctypes.POINTER(mfa_launch_config)], _I),
    "mfa_form_set_config": ([_VP, ctypes.POINTER(mfa_launch_config)], _I),
    "mfa_form_autotune": ([_VP, _VP, _VP, _VP, _I, _VP, _I, ctypes.POINTER(_I)], _I),
    "mfa_apply": ([_VP, _VP, _VP, _VP, _I], _I),
    "mfa_apply_host": ([_VP, _VP, _VP, _VP], _I),
    "mfa_apply_host_many": ([_VP, _I, _VP, _VP, _VP], _I),
    "mfa_apply_f32": ([_VP, _VP, _VP, _VP, _I], _I),
    "mfa_convert_f64_to_f32": ([_VP, _VP, _VP, _I64], _I),
    "mfa_convert_f32_to_f64": ([_VP, _VP, _VP, _I64], _I),
    "mfa_sync": ([_VP], _I),
    "mfa_diagonal": ([_VP, _VP, _VP], _I),
    "mfa_cg": ([_VP, _VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "mfa_fcg_mixed": ([_VP, _VP, _VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                       ctypes.POINTER(_D)], _I),
    "mfa_fcg_learned": ([_VP, _VP, _VP, _VP, _I, _VP, _VP, _D, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                         ctypes.POINTER(_D), ctypes.POINTER(_I)], _I),
    "mfa_probe_fp64_fma": ([_VP, ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "mfa_halo_pack": ([_VP, _VP, _I64, _I, _I64, _VP, _VP], _I),
    "mfa_halo_unpack": ([_VP, _VP, _I64, _I, _I64, _VP, _VP, _I], _I),
    "mfa_precond_create": ([_VP, _VP, _I, ctypes.c_uint64, _PP], _I),
    "mfa_precond_apply": ([_VP, _VP, _VP, _VP], _I),
    "mfa_precond_loss_grad": ([_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_D), _VP], _I),
    "mfa_precond_train": ([_VP, _VP, _VP, _I, _VP, _VP, _I, _D, ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "mfa_precond_get_weights": ([_VP, _VP], _I),
    "mfa_precond_set_weights": ([_VP, _VP], _I),
    "mfa_precond_save": ([_VP, ctypes.c_char_p], _I),
    "mfa_precond_load": ([_VP, ctypes.c_char_p], _I),
    "mfa_precond_destroy": ([_VP], _I),
    "mfa_apply_batched": ([_VP, _I, _VP, _VP, _VP], _I),
    "mfa_batch_create": ([_VP, _I, _VP, _VP, _VP, _PP], _I),
    "mfa_batch_apply": ([_VP, _VP], _I),
    "mfa_batch_info": ([_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "mfa_batch_destroy": ([_VP], _I),
    "mfa_order_rcm": ([_I64, _I, _VP, _I64, _I, _VP, _I64, _VP, _VP], _I),
    "mfa_cg_noalloc": ([_VP, _VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
}
MFA_CG_NOALLOC_MAX_NDOF = 262144
MFA_PRECOND_NPARAMS = 32896


def lib():
    """Load libmfa.so (built by ``build()``); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmfa.so not found at %s: run paper_1903_08243_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != MFA_OK:
        raise MfaError(rc, lib().mfa_last_error().decode())


def _ptr(a):
    """Address of a numpy array or a torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- the C ABI under the same names (status codes become MfaError)

def mfa_create(device=0, stream=None):
    h = ctypes.c_void_p()
    _check(lib().mfa_create(ctypes.byref(h), device, _stream_handle(stream)))
    return h


def mfa_set_stream(ctx, stream):
    _check(lib().mfa_set_stream(ctx, _stream_handle(stream)))


def mfa_destroy(ctx):
    _check(lib().mfa_destroy(ctx))


def mfa_mesh_upload(ctx, cell_type, coords, cell_vert):
    coords = np.ascontiguousarray(coords, dtype=np.float64)
    cell_vert = np.ascontiguousarray(cell_vert, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().mfa_mesh_upload(ctx, cell_type, cell_vert.shape[0], coords.shape[0], _ptr(coords), _ptr(cell_vert),
                                 ctypes.byref(h)))
    return h


def mfa_mesh_destroy(mesh):
    _check(lib().mfa_mesh_destroy(mesh))


def mfa_space_create(ctx, mesh, degree, ncomp, cell_node=None, nnode=0):
    """cell_node None: the library builds the map from the mesh."""
    if cell_node is not None:
        cell_node = np.ascontiguousarray(cell_node, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().mfa_space_create(ctx, mesh, degree, ncomp, _ptr(cell_node), int(nnode), ctypes.byref(h)))
    return h


def mfa_space_ndof(space):
    n = ctypes.c_int64()
    _check(lib().mfa_space_ndof(space, ctypes.byref(n)))
    return n.value


def mfa_space_destroy(space):
    _check(lib().mfa_space_destroy(space))


def mfa_form_create(ctx, space, params):
    h = ctypes.c_void_p()
    _check(lib().mfa_form_create(ctx, space, ctypes.byref(params), ctypes.byref(h)))
    return h


def mfa_form_set_coefficient(form, u):
    _check(lib().mfa_form_set_coefficient(form, _ptr(u)))


def mfa_form_get_info(form):
    info = mfa_form_info()
    _check(lib().mfa_form_get_info(form, ctypes.byref(info)))
    return info


def mfa_form_destroy(form):
    _check(lib().mfa_form_destroy(form))


def _nloc(cell_type, degree):
    if cell_type == MFA_CELL_HEX8:
        return (degree + 1) ** 3
    if cell_type == MFA_CELL_QUAD4:
        return (degree + 1) ** 2
    if cell_type == MFA_CELL_TRI3:
        return (degree + 1) * (degree + 2) // 2
    return {1: 4, 2: 10}.get(degree, (degree + 1) * (degree + 2) * (degree + 3) // 6)


def mfa_build_cell_node(cell_type, degree, cell_vert, nvert):
    """Conforming cell -> node map from the vertex connectivity (host): returns (cell_node, nnode)."""
    cv = np.ascontiguousarray(cell_vert, dtype=np.int32)
    cn = np.empty((cv.shape[0], _nloc(cell_type, degree)), dtype=np.int32)
    nn = ctypes.c_int64()
    _check(lib().mfa_build_cell_node(cell_type, degree, cv.shape[0], cv.ctypes.data, int(nvert), cn.ctypes.data,
                                     ctypes.byref(nn)))
    return cn, nn.value


def mfa_node_coords(cell_type, degree, cell_vert, coords, cell_node, nnode):
    cv = np.ascontiguousarray(cell_vert, dtype=np.int32)
    X = np.ascontiguousarray(coords, dtype=np.float64)
    cn = np.ascontiguousarray(cell_node, dtype=np.int32)
    out = np.empty((int(nnode), 3))
    _check(lib().mfa_node_coords(cell_type, degree, cv.shape[0], cv.ctypes.data, X.ctypes.data, cn.ctypes.data,
                                 int(nnode), out.ctypes.data))
    return out


def mfa_simplex_rule(cell_type, degree):
    """The library's fully symmetric simplex rule of `degree`: (points [nq][dim], weights [nq])."""
    dim = 2 if cell_type == MFA_CELL_TRI3 else 3
    pts, w, n = np.empty((24, dim)), np.empty(24), ctypes.c_int()
    _check(lib().mfa_simplex_rule(cell_type, degree, 24, pts.ctypes.data, w.ctypes.data, ctypes.byref(n)))
    return pts[:n.value].copy(), w[:n.value].copy()


def mfa_space_get_cell_node(space, ncell, nloc):
    out = np.empty((ncell, nloc), dtype=np.int32)
    _check(lib().mfa_space_get_cell_node(space, out.ctypes.data))
    return out


def mfa_order_rcm(cell_vert, cell_node, nnode, nvert=None):
    """Reverse Cuthill-McKee renumbering (host): returns (cell_order, node_perm) with
    cell_order[new] = old cell and node_perm[old] = new node."""
    cv = np.ascontiguousarray(cell_vert, dtype=np.int32)
    cn = np.ascontiguousarray(cell_node, dtype=np.int32)
    ncell, nv = cv.shape
    nloc = cn.shape[1]
    if nvert is None:
        nvert = int(cv.max()) + 1 if cv.size else 0
    cell_order = np.empty(ncell, dtype=np.int32)
    node_perm = np.empty(int(nnode), dtype=np.int32)
    _check(lib().mfa_order_rcm(ncell, nv, cv.ctypes.data, int(nvert), nloc, cn.ctypes.data, int(nnode),
                               cell_order.ctypes.data, node_perm.ctypes.data))
    return cell_order, node_perm


def apply_order(cell_vert, cell_node, cell_order, node_perm):
    """Maps in the new numbering: cells in cell_order, node ids through node_perm."""
    cv = np.ascontiguousarray(np.asarray(cell_vert)[cell_order])
    cn = np.ascontiguousarray(node_perm[np.asarray(cell_node)[cell_order]]).astype(np.int32)
    return cv, cn


def mfa_form_set_dirichlet(form, dofs):
    d = np.ascontiguousarray(dofs, dtype=np.int32)
    _check(lib().mfa_form_set_dirichlet(form, d.ctypes.data if d.size else None, d.size))


def mfa_form_list_configs(form):
    n = ctypes.c_int()
    _check(lib().mfa_form_list_configs(form, None, 0, ctypes.byref(n)))
    arr = (mfa_launch_config * max(n.value, 1))()
    _check(lib().mfa_form_list_configs(form, arr, n.value, ctypes.byref(n)))
    return [arr[i] for i in range(n.value)]


def mfa_form_get_config(form):
    c = mfa_launch_config()
    _check(lib().mfa_form_get_config(form, ctypes.byref(c)))
    return c


def mfa_form_set_config(form, cfg):
    _check(lib().mfa_form_set_config(form, ctypes.byref(cfg)))


def mfa_form_autotune(ctx, form, x, y, reps=3):
    """Time every configuration, keep the fastest; returns the list with times."""
    n = ctypes.c_int()
    _check(lib().mfa_form_list_configs(form, None, 0, ctypes.byref(n)))
    arr = (mfa_launch_config * max(n.value, 1))()
    _check(lib().mfa_form_autotune(ctx, form, _ptr(x), _ptr(y), reps, arr, n.value, ctypes.byref(n)))
    return [arr[i] for i in range(n.value)]


def mfa_apply(ctx, form, x, y, accumulate=False):
    _check(lib().mfa_apply(ctx, form, _ptr(x), _ptr(y), int(accumulate)))


def mfa_apply_f32(ctx, form, x, y, accumulate=False):
    _check(lib().mfa_apply_f32(ctx, form, _ptr(x), _ptr(y), int(accumulate)))


def mfa_probe_fp64_fma(ctx):
    """Measured FP64 FMA throughput: (TFLOP/s, median SM MHz during the probe)."""
    t, f = ctypes.c_double(), ctypes.c_double()
    _check(lib().mfa_probe_fp64_fma(ctx, ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def mfa_halo_pack(ctx, ids, ncomp, nnode, v, buf):
    """buf[k] = v[ids[k]] (device tensors: ids int32, v and buf float64, ncomp values per node)."""
    _check(lib().mfa_halo_pack(ctx, _ptr(ids), ids.numel(), ncomp, nnode, _ptr(v), _ptr(buf)))


def mfa_halo_unpack(ctx, ids, ncomp, nnode, buf, v, accumulate=False):
    """v[ids[k]] = buf[k] (or += with accumulate)."""
    _check(lib().mfa_halo_unpack(ctx, _ptr(ids), ids.numel(), ncomp, nnode, _ptr(buf), _ptr(v), int(accumulate)))


def mfa_convert_f64_to_f32(ctx, x, y):
    _check(lib().mfa_convert_f64_to_f32(ctx, _ptr(x), _ptr(y), x.numel()))


def mfa_convert_f32_to_f64(ctx, x, y):
    _check(lib().mfa_convert_f32_to_f64(ctx, _ptr(x), _ptr(y), x.numel()))


def mfa_apply_host(ctx, form, x_host, y_host):
    _check(lib().mfa_apply_host(ctx, form, _ptr(x_host), _ptr(y_host)))


def mfa_apply_host_many(ctx, forms, xs_host, ys_host):
    """ys_host[i] = A_i xs_host[i] with the host<->device copies overlapped with the applies (host tensors, best
    pinned)."""
    n = len(forms)
    if len(xs_host) != n or len(ys_host) != n:
        raise ValueError("one x and one y per form")
    fa = (ctypes.c_void_p * max(n, 1))(*[f for f in forms])
    xa = (ctypes.c_void_p * max(n, 1))(*[_ptr(x) for x in xs_host])
    ya = (ctypes.c_void_p * max(n, 1))(*[_ptr(y) for y in ys_host])
    _check(lib().mfa_apply_host_many(ctx, n, fa, xa, ya))


def mfa_sync(ctx):
    _check(lib().mfa_sync(ctx))


def mfa_diagonal(ctx, form, d):
    _check(lib().mfa_diagonal(ctx, form, _ptr(d)))


def mfa_cg(ctx, form, precond, b, x, rtol, maxit):
    """Returns (status, iterations, relative residual); raises on errors other than non-convergence."""
    it, rel = ctypes.c_int(), ctypes.c_double()
    rc = lib().mfa_cg(ctx, form, precond, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(it), ctypes.byref(rel))
    if rc not in (MFA_OK, MFA_ERR_NOT_CONVERGED):
        _check(rc)
    return rc, it.value, rel.value


def mfa_fcg_mixed(ctx, outer, inner, inner_iters, b, x, rtol, maxit):
    """Returns (status, outer iterations, inner iterations, relative residual)."""
    it, inn, rel = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    rc = lib().mfa_fcg_mixed(ctx, outer, inner, inner_iters, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(it),
                             ctypes.byref(inn), ctypes.byref(rel))
    if rc not in (MFA_OK, MFA_ERR_NOT_CONVERGED):
        _check(rc)
    return rc, it.value, inn.value, rel.value


def mfa_fcg_learned(ctx, outer, inner, pc, inner_iters, b, x, rtol, maxit, fallback=True, raise_on_breakdown=True):
    """Returns (status, outer iterations, inner iterations, relative residual, used_fallback)."""
    it, inn, rel, fb = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    rc = lib().mfa_fcg_learned(ctx, outer, inner, pc, inner_iters, _ptr(b), _ptr(x), rtol, maxit, int(fallback),
                               ctypes.byref(it), ctypes.byref(inn), ctypes.byref(rel), ctypes.byref(fb))
    ok = (MFA_OK, MFA_ERR_NOT_CONVERGED) if raise_on_breakdown else (MFA_OK, MFA_ERR_NOT_CONVERGED, MFA_ERR_BREAKDOWN)
    if rc not in ok:
        _check(rc)
    return rc, it.value, inn.value, rel.value, fb.value


def mfa_precond_create(ctx, form, seed=0, mode=0):
    h = ctypes.c_void_p()
    _check(lib().mfa_precond_create(ctx, form, mode, seed, ctypes.byref(h)))
    return h


def mfa_precond_apply(ctx, pc, r, z):
    _check(lib().mfa_precond_apply(ctx, pc, _ptr(r), _ptr(z)))


def mfa_precond_loss_grad(ctx, pc, aform, r, e, want_grad=True):
    loss = ctypes.c_double()
    g = np.zeros(MFA_PRECOND_NPARAMS, dtype=np.float32) if want_grad else None
    _check(lib().mfa_precond_loss_grad(ctx, pc, aform, _ptr(r), _ptr(e), ctypes.byref(loss), _ptr(g)))
    return loss.value, g


def mfa_precond_train(ctx, pc, aform, rs, es, steps, lr):
    first, last = ctypes.c_double(), ctypes.c_double()
    _check(lib().mfa_precond_train(ctx, pc, aform, len(rs), _ptr_array(rs), _ptr_array(es), steps, lr,
                                   ctypes.byref(first), ctypes.byref(last)))
    return first.value, last.value


def mfa_precond_get_weights(pc):
    w = np.zeros(MFA_PRECOND_NPARAMS, dtype=np.float32)
    _check(lib().mfa_precond_get_weights(pc, _ptr(w)))
    return w


def mfa_precond_set_weights(pc, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    _check(lib().mfa_precond_set_weights(pc, _ptr(w)))


def mfa_precond_save(pc, path):
    _check(lib().mfa_precond_save(pc, str(path).encode()))


def mfa_precond_load(pc, path):
    _check(lib().mfa_precond_load(pc, str(path).encode()))


def mfa_precond_destroy(pc):
    _check(lib().mfa_precond_destroy(pc))


def unpack_precond_weights(w, nloc):
    """(W1 [128][nloc], b1 [128], W2 [nloc][128]) from the master layout."""
    W1 = w[:128 * 128].reshape(128, 128)[:, :nloc]
    b1 = w[128 * 128:128 * 128 + 128]
    W2 = w[128 * 128 + 128:].reshape(128, 128)[:nloc, :]
    return W1, b1, W2


def pack_precond_weights(W1, b1, W2):
    w = np.zeros(MFA_PRECOND_NPARAMS, dtype=np.float32)
    nloc = W1.shape[1]
    w[:128 * 128].reshape(128, 128)[:, :nloc] = W1
    w[128 * 128:128 * 128 + 128] = b1
    w[128 * 128 + 128:].reshape(128, 128)[:nloc, :] = W2
    return w


def _ptr_array(items, ctype=ctypes.c_void_p):
    arr = (ctype * max(1, len(items)))()
    for i, it in enumerate(items):
        arr[i] = it if isinstance(it, int) or it is None else (it.value if isinstance(it, ctypes.c_void_p) else _ptr(it))
    return arr


def mfa_apply_batched(ctx, forms, xs, ys):
    fa = _ptr_array([f.value for f in forms])
    _check(lib().mfa_apply_batched(ctx, len(forms), fa, _ptr_array(xs), _ptr_array(ys)))


def mfa_batch_create(ctx, forms, xs, ys):
    h = ctypes.c_void_p()
    fa = _ptr_array([f.value for f in forms])
    _check(lib().mfa_batch_create(ctx, len(forms), fa, _ptr_array(xs), _ptr_array(ys), ctypes.byref(h)))
    return h


def mfa_batch_apply(ctx, batch):
    _check(lib().mfa_batch_apply(ctx, batch))


def mfa_batch_info(batch):
    g, s = ctypes.c_int(), ctypes.c_int()
    _check(lib().mfa_batch_info(batch, ctypes.byref(g), ctypes.byref(s)))
    return g.value, s.value


def mfa_batch_destroy(batch):
    _check(lib().mfa_batch_destroy(batch))


def mfa_cg_noalloc(ctx, form, precond, b, x, rtol, maxit):
    """mfa_cg without device allocation (work vectors in a fixed device array,
    at most MFA_CG_NOALLOC_MAX_NDOF dofs).  Returns (status, iterations, relative
    residual); raises on errors other than non-convergence."""
    it, rel = ctypes.c_int(), ctypes.c_double()
    rc = lib().mfa_cg_noalloc(ctx, form, precond, _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(it), ctypes.byref(rel))
    if rc not in (MFA_OK, MFA_ERR_NOT_CONVERGED):
        _check(rc)
    return rc, it.value, rel.value


# ---- small owning wrappers (destroy in reverse order of creation)

class Context:
    def __init__(self, device=0, stream=None):
        self.h = mfa_create(device, stream)

    def sync(self):
        mfa_sync(self.h)

    def close(self):
        if self.h:
            mfa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx, cell_type, coords, cell_vert):
        self.ctx = ctx
        self.cell_type = cell_type
        self.ncell = int(np.asarray(cell_vert).shape[0])
        self.nvert = int(np.asarray(coords).shape[0])
        self.h = mfa_mesh_upload(ctx.h, cell_type, coords, cell_vert)

    def __del__(self):
        try:
            if self.h:
                mfa_mesh_destroy(self.h)
        except Exception:
            pass


class Space:
    def __init__(self, mesh, degree, ncomp, cell_node=None, nnode=0):
        self.mesh = mesh
        self.degree, self.ncomp = degree, ncomp
        self.h = mfa_space_create(mesh.ctx.h, mesh.h, degree, ncomp, cell_node, nnode)
        self.ndof = mfa_space_ndof(self.h)
        self.nnode = self.ndof // ncomp

    def cell_node(self):
        return mfa_space_get_cell_node(self.h, self.mesh.ncell, _nloc(self.mesh.cell_type, self.degree))

    def __del__(self):
        try:
            if self.h:
                mfa_space_destroy(self.h)
        except Exception:
            pass


def form_params(kind, law=MFA_LAW_SVK, qdeg=0, precision=MFA_PREC_FP64, scatter=MFA_SCATTER_AUTO, k2=1.0,
                lam=1.0, mu=1.0, b=(0.0, 0.0, 0.0), cells_per_block=0, geometry=MFA_GEOM_STORED, rule=MFA_RULE_AUTO):
    p = mfa_form_params()
    p.kind, p.law, p.qdeg, p.precision, p.scatter = kind, law, qdeg, precision, scatter
    p.cells_per_block, p.geometry, p.rule = cells_per_block, geometry, rule
    p.k2, p.lam, p.mu = k2, lam, mu
    p.b[0], p.b[1], p.b[2] = b
    return p


class Form:
    def __init__(self, space, kind, **kw):
        self.space = space
        self.ctx = space.mesh.ctx
        self.params = form_params(kind, **kw)
        self.h = mfa_form_create(self.ctx.h, space.h, self.params)
        self._coef = None

    def info(self):
        return mfa_form_get_info(self.h)

    def set_dirichlet(self, dofs):
        mfa_form_set_dirichlet(self.h, dofs)

    def configs(self):
        return mfa_form_list_configs(self.h)

    def config(self):
        return mfa_form_get_config(self.h)

    def set_config(self, cfg):
        mfa_form_set_config(self.h, cfg)

    def set_max_blocks(self, k):
        """Cap the persistent grid of this form's launches at k blocks (0: one wave per SM)."""
        cfg = mfa_form_get_config(self.h)
        cfg.max_blocks = int(k)
        mfa_form_set_config(self.h, cfg)

    def autotune(self, x, y, reps=3):
        return mfa_form_autotune(self.ctx.h, self.h, x, y, reps)

    def set_coefficient(self, u):
        self._coef = u  # keep the borrowed buffer alive
        mfa_form_set_coefficient(self.h, u)

    def apply(self, x, y=None, accumulate=False):
        if y is None:
            import torch

            y = torch.empty_like(x)
        mfa_apply(self.ctx.h, self.h, x, y, accumulate)
        return y

    def apply_host(self, x_host, y_host=None):
        x_host = np.ascontiguousarray(x_host, dtype=np.float64)
        if y_host is None:
            y_host = np.empty_like(x_host)
        mfa_apply_host(self.ctx.h, self.h, x_host, y_host)
        return y_host

    def diagonal(self, d=None):
        if d is None:
            import torch

            d = torch.empty(self.space.ndof, dtype=torch.float64, device="cuda")
        mfa_diagonal(self.ctx.h, self.h, d)
        return d

    def cg(self, b, x, precond=MFA_PC_JACOBI, rtol=1e-8, maxit=10000):
        return mfa_cg(self.ctx.h, self.h, precond, b, x, rtol, maxit)

    def __del__(self):
        try:
            if self.h:
                mfa_form_destroy(self.h)
        except Exception:
            pass
