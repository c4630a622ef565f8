"""GPU parity of the planar cells (Table 2's tri and quad columns) against the FP64 oracle: quadrilaterals Q1-Q8
(sum-factorised, p+1 / p+2 / 2p+2 points) and triangles P1-P6 (one thread per cell for P1-P4, one warp per cell for
every degree), every form; vector forms in plane strain."""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
from tests.problems import KIND_NAMES, oracle_problem, quad_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

TOL = 1e-12
VECTOR = [("laplace", 0), ("elasticity", 0), ("hyper_res", mfa.MFA_LAW_SVK), ("hyper_res", mfa.MFA_LAW_NEOHOOKE),
          ("hyper_jac", mfa.MFA_LAW_SVK), ("hyper_jac", mfa.MFA_LAW_NEOHOOKE)]


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


FORM_ONLY = ("scatter", "precision", "geometry", "cells_per_block")


def run_check(ctx, case, kind, x, u=None, qdeg=None, **kw):
    okw = {k: v for k, v in kw.items() if k not in FORM_ONLY}
    ref = oracle_problem(case, kind, qdeg=qdeg, ucoef=u if kind == "hyper_jac" else None, **okw).apply(x)
    form = make_form(ctx, case, kind, qdeg=qdeg or 0, **kw)
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    y = y.cpu().numpy()
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    mx = np.abs(y - ref).max() / np.abs(ref).max()
    assert rel <= TOL and mx <= TOL, (rel, mx)
    return form


def vec_inputs(case, kind, seed):
    u = fi.sinusoid_displacement(case["nodes"], seed=seed)[:, :2].ravel()
    x = u if kind == "hyper_res" else fi.uniform_vector(u.size, seed=seed + 50)
    return u, x


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("scatter", [mfa.MFA_SCATTER_ATOMIC, mfa.MFA_SCATTER_COLOUR])
def test_quad_scalar(ctx, p, kind, scatter):
    case = quad_case({1: 17, 2: 11, 3: 9, 4: 7, 6: 5, 8: 4}[p], p)
    x = fi.uniform_vector(case["nnode"], seed=p)
    f = run_check(ctx, case, kind, x, k2=0.8, scatter=scatter)
    assert f.config().variant == mfa.MFA_VARIANT_POINT
    # one kernel, atomic or colour scatter (no warp-aggregated one for quads)
    assert sorted(c.scatter for c in f.configs()) == sorted([mfa.MFA_SCATTER_ATOMIC, mfa.MFA_SCATTER_COLOUR])


@pytest.mark.parametrize("p", [1, 3, 6])
def test_quad_scalar_p_plus_2(ctx, p):
    case = quad_case(6, p)
    run_check(ctx, case, "helmholtz", fi.uniform_vector(case["nnode"], seed=9), qdeg=p + 2, k2=0.8)


@pytest.mark.parametrize("p", [1, 2, 4])
@pytest.mark.parametrize("kind, law", VECTOR)
def test_quad_vector(ctx, p, kind, law):
    case = quad_case({1: 9, 2: 7, 4: 5}[p], p, ncomp=2)
    u, x = vec_inputs(case, kind, seed=10 + p)
    kw = dict(lam=1.3, mu=0.7, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.1, -0.2, 0.0)
    run_check(ctx, case, kind, x, u, **kw)


@pytest.mark.parametrize("p, kind, law", [(1, "elasticity", 0), (3, "elasticity", 0), (2, "hyper_res", 1),
                                          (2, "hyper_jac", 0), (4, "hyper_jac", 1)])
def test_quad_table2_rules(ctx, p, kind, law):
    qdeg = 2 * p + 2 if kind.startswith("hyper") else p + 2
    case = quad_case(5, p, ncomp=2)
    u, x = vec_inputs(case, kind, seed=30 + p)
    run_check(ctx, case, kind, x, u, qdeg=qdeg, lam=1.0, mu=1.0, law=law)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
def test_tri_scalar(ctx, p, kind):
    case = tri_case({1: 12, 2: 8, 3: 6, 4: 5, 5: 4, 6: 4}[p], p)
    f = run_check(ctx, case, kind, fi.uniform_vector(case["nnode"], seed=40 + p), k2=0.6,
                  scatter=mfa.MFA_SCATTER_COLOUR if p % 2 else mfa.MFA_SCATTER_ATOMIC)
    assert f.config().variant == (mfa.MFA_VARIANT_CELL if p <= 4 else mfa.MFA_VARIANT_CELL_WARP)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
@pytest.mark.parametrize("kind, law", VECTOR)
def test_tri_vector(ctx, p, kind, law):
    case = tri_case(4, p, ncomp=2, seed=5)
    u, x = vec_inputs(case, kind, seed=50 + p)
    kw = dict(lam=1.2, mu=0.9, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.05, 0.1, 0.0)
    run_check(ctx, case, kind, x, u, **kw)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind, law, ncomp", [("mass", 0, 1), ("laplace", 0, 1), ("helmholtz", 0, 1)] +
                         [(k, law, 2) for k, law in VECTOR])
def test_tri_every_config(ctx, p, kind, law, ncomp):
    """P1-P4 have two kernels (one thread per cell, the default, and one warp per cell; the P4 Jacobian action only
    the second): every configuration the form lists, thread counts and scatters included, gives the oracle's
    result."""
    case = tri_case(5, p, ncomp=ncomp, seed=9)
    if ncomp == 1:
        u, x = None, fi.uniform_vector(case["nnode"], seed=70 + p)
        kw = dict(k2=0.6)
    else:
        u, x = vec_inputs(case, kind, seed=70 + p)
        kw = dict(lam=1.2, mu=0.9, law=law, b=(0.05, 0.1, 0.0))
    okw = dict(kw) if ncomp == 2 and kind == "hyper_res" else {k: v for k, v in kw.items() if k != "b"}
    ref = oracle_problem(case, kind, ucoef=u if kind == "hyper_jac" else None, **okw).apply(x)
    form = make_form(ctx, case, kind, **okw)
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    cfgs = form.configs()
    variants = {c.variant for c in cfgs}
    if p == 4 and kind == "hyper_jac":
        assert variants == {mfa.MFA_VARIANT_CELL_WARP}
    else:
        assert variants == {mfa.MFA_VARIANT_CELL, mfa.MFA_VARIANT_CELL_WARP}
        assert {c.cells_per_block for c in cfgs if c.variant == mfa.MFA_VARIANT_CELL} == {32, 64, 128}
    assert all(c.scatter != mfa.MFA_SCATTER_WARP for c in cfgs)
    xd = torch.from_numpy(x).cuda()
    for c in cfgs:
        form.set_config(c)
        y = form.apply(xd)
        ctx.sync()
        y = y.cpu().numpy()
        rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert rel <= TOL and np.abs(y - ref).max() <= TOL * np.abs(ref).max(), (c.as_dict(), rel)
    yd = torch.empty_like(xd)
    best = form.autotune(xd, yd)
    assert form.config().variant in variants and best is not None


@pytest.mark.parametrize("cell, p", [("quad", 3), ("tri", 4)])
def test_planar_library_built_map_and_cg(ctx, cell, p):
    mesh = fi.quad_mesh(6, perturb=0.1, seed=3) if cell == "quad" else fi.tri_mesh(6, perturb=0.1, seed=3)
    ct = mfa.MFA_CELL_QUAD4 if cell == "quad" else mfa.MFA_CELL_TRI3
    m = mfa.Mesh(ctx, ct, mesh.coords, mesh.cell_vert)
    sp = mfa.Space(m, p, 1)
    cn = sp.cell_node()
    A = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, k2=1.0)
    pb = oracle.Problem(3 if cell == "tri" else 40, mesh.coords, mesh.cell_vert, p, cn, sp.nnode, 2,
                        qdeg=p + 1 if cell == "quad" else 2 * p)
    x = fi.uniform_vector(sp.ndof, seed=60)
    y = A.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    ref = pb.apply(x)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= TOL
    b = torch.from_numpy(ref).cuda()
    u = torch.zeros_like(b)
    rc, it, rel = mfa.mfa_cg(ctx.h, A.h, mfa.MFA_PC_NONE, b, u, 1e-12, 2000)
    assert rc == mfa.MFA_OK
    assert np.linalg.norm(u.cpu().numpy() - x) / np.linalg.norm(x) <= 1e-8


def test_planar_limits(ctx):
    case = quad_case(3, 2)
    for kw in [dict(precision=mfa.MFA_PREC_FP32), dict(scatter=mfa.MFA_SCATTER_WARP),
               dict(geometry=mfa.MFA_GEOM_ONTHEFLY)]:
        with pytest.raises(mfa.MfaError) as e:
            make_form(ctx, case, "helmholtz", **kw)
        assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    with pytest.raises(mfa.MfaError):
        make_form(ctx, case, "elasticity")  # a scalar space
