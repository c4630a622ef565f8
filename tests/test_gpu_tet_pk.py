"""GPU parity of the P3..P6 tet kernel (dense tabulation, one warp per cell) against the FP64 oracle: every form,
both scatters, chunked quadrature with ragged last chunks (27..343 points per cell)."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, assembled_dense, oracle_problem, tet_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

TOL = 1e-12
SCALAR = ["mass", "laplace", "helmholtz"]
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


def check(y, ref):
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    mx = np.abs(y - ref).max() / np.abs(ref).max()
    assert rel <= TOL and mx <= TOL, (rel, mx)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
@pytest.mark.parametrize("kind", SCALAR)
@pytest.mark.parametrize("scatter", [mfa.MFA_SCATTER_ATOMIC, mfa.MFA_SCATTER_COLOUR])
def test_tet_pk_scalar_parity(ctx, p, kind, scatter):
    case = tet_case(3 if p <= 4 else 2, p, perturb=0.15, seed=p)
    x = fi.uniform_vector(case["nnode"], seed=40 + p)
    ref = oracle_problem(case, kind, k2=0.7).apply(x)
    form = make_form(ctx, case, kind, k2=0.7, scatter=scatter)
    # one thread per cell where the rule has at most 24 points (Table 2's symmetric rules: P3 every scalar form,
    # P4 Laplace), else one warp per cell; every listed configuration gives the oracle's result
    cell = p == 3 or (p == 4 and kind == "laplace")
    assert form.config().variant == (mfa.MFA_VARIANT_CELL if cell else mfa.MFA_VARIANT_CELL_WARP)
    variants = {c.variant for c in form.configs()}
    assert variants == ({mfa.MFA_VARIANT_CELL, mfa.MFA_VARIANT_CELL_WARP} if cell else {mfa.MFA_VARIANT_CELL_WARP})
    xd = torch.from_numpy(x).cuda()
    for c in form.configs():
        form.set_config(c)
        y = form.apply(xd)
        ctx.sync()
        check(y.cpu().numpy(), ref)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
@pytest.mark.parametrize("kind, law", VECTOR)
def test_tet_pk_vector_parity(ctx, p, kind, law):
    case = tet_case(2, p, ncomp=3, perturb=0.15, seed=10 + p)
    u = fi.sinusoid_displacement(case["nodes"], seed=p).ravel()
    x = u if kind == "hyper_res" else fi.uniform_vector(u.size, seed=60 + p)
    kw = dict(lam=1.3, mu=0.7, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.1, -0.2, 0.05)
    ref = oracle_problem(case, kind, ucoef=u if kind == "hyper_jac" else None, **kw).apply(x)
    form = make_form(ctx, case, kind, **kw)
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    check(y.cpu().numpy(), ref)


def test_tet_pk_shuffled_numbering_and_cg(ctx):
    case = tet_case(2, 4, perturb=0.1, seed=3, shuffle=True)
    x = fi.uniform_vector(case["nnode"], seed=70)
    pb = oracle_problem(case, "helmholtz")
    form = make_form(ctx, case, "helmholtz")
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    check(y.cpu().numpy(), pb.apply(x))
    # the Helmholtz operator is SPD: plain CG reaches the dense solution
    A = assembled_dense(pb, case)
    b = fi.uniform_vector(case["nnode"], seed=71)
    bd = torch.from_numpy(b).cuda()
    xs = torch.zeros_like(bd)
    rc, it, rel = mfa.mfa_cg(ctx.h, form.h, mfa.MFA_PC_NONE, bd, xs, 1e-12, 5000)
    assert rc == mfa.MFA_OK
    u_ref = np.linalg.solve(A, b)
    assert np.linalg.norm(xs.cpu().numpy() - u_ref) / np.linalg.norm(u_ref) <= 1e-9


def test_tet_pk_unsupported_paths(ctx):
    case = tet_case(2, 3)
    with pytest.raises(mfa.MfaError) as e:
        make_form(ctx, case, "helmholtz", scatter=mfa.MFA_SCATTER_WARP)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    form = make_form(ctx, tet_case(2, 3, ncomp=3), "hyper_res", law=mfa.MFA_LAW_SVK)
    with pytest.raises(mfa.MfaError) as e:  # the diagonal covers the linear forms (test_gpu_diag.py)
        form.diagonal()
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
