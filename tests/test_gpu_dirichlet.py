"""Dirichlet constraints: the constrained action R A R x + (I - R) x against the oracle, the diagonal, and
clamped-elasticity CG against a dense solve of the oracle's assembled matrix."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, hex_case, oracle_problem, quad_case, tet_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def clamped_dofs(case):
    nc = case["ncomp"]
    fixed = np.flatnonzero(case["nodes"][:, 0] < 1e-12)
    return (nc * fixed[:, None] + np.arange(nc)[None, :]).ravel()


PLANAR = {"quad": lambda seed: quad_case(3, 2, ncomp=2, seed=seed), "tri": lambda seed: tri_case(3, 3, ncomp=2, seed=seed)}


def constrained(pb, x, dofs):
    r = np.ones(x.size)
    r[dofs] = 0.0
    return r * pb.apply(r * x) + (1.0 - r) * x


@pytest.mark.parametrize("cell", ["tet", "hex", "quad", "tri"])
def test_constrained_action_matches_the_definition(ctx, cell):
    if cell in PLANAR:
        case = PLANAR[cell](2)
    else:
        case = tet_case(3, 2, ncomp=3, perturb=0.1, seed=2) if cell == "tet" else hex_case(3, 2, ncomp=3)
    dofs = clamped_dofs(case)
    x = fi.uniform_vector(case["nnode"] * case["ncomp"], seed=21)
    ref = constrained(oracle_problem(case, "elasticity", lam=1.2, mu=0.8), x, dofs)
    form = make_form(ctx, case, "elasticity", lam=1.2, mu=0.8)
    form.set_dirichlet(dofs)
    xd = torch.from_numpy(x).cuda()
    y = form.apply(xd)
    ctx.sync()
    y = y.cpu().numpy()
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 1e-12
    np.testing.assert_array_equal(y[dofs], x[dofs])
    # accumulate: y += A_D x
    y2 = torch.from_numpy(y).cuda()
    mfa.mfa_apply(ctx.h, form.h, xd, y2, True)
    ctx.sync()
    assert np.linalg.norm(y2.cpu().numpy() - 2 * ref) / np.linalg.norm(ref) <= 1e-12
    # removing the constraints gives the plain operator back
    form.set_dirichlet([])
    y3 = form.apply(xd)
    ctx.sync()
    ref3 = oracle_problem(case, "elasticity", lam=1.2, mu=0.8).apply(x)
    assert np.linalg.norm(y3.cpu().numpy() - ref3) / np.linalg.norm(ref3) <= 1e-12


def test_constrained_diagonal(ctx):
    case = tet_case(2, 2, ncomp=3, perturb=0.1, seed=3)
    dofs = clamped_dofs(case)
    pb = oracle_problem(case, "elasticity")
    ref = np.diag(pb.dense()).copy()
    ref[dofs] = 1.0
    form = make_form(ctx, case, "elasticity")
    form.set_dirichlet(dofs)
    d = form.diagonal()
    ctx.sync()
    np.testing.assert_allclose(d.cpu().numpy(), ref, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("cell, precond", [("tet", mfa.MFA_PC_JACOBI), ("tet", mfa.MFA_PC_NONE),
                                           ("hex", mfa.MFA_PC_NONE), ("hex", mfa.MFA_PC_JACOBI),
                                           ("quad", mfa.MFA_PC_JACOBI), ("tri", mfa.MFA_PC_JACOBI)])
def test_clamped_elasticity_cg_matches_dense_solve(ctx, cell, precond):
    if cell in PLANAR:
        case = PLANAR[cell](4)
    else:
        case = tet_case(2, 2, ncomp=3, perturb=0.1, seed=4) if cell == "tet" else hex_case(2, 2, ncomp=3)
    dofs = clamped_dofs(case)
    pb = oracle_problem(case, "elasticity")
    A = pb.dense()
    r = np.ones(pb.ndof)
    r[dofs] = 0.0
    AD = r[:, None] * A * r[None, :] + np.diag(1.0 - r)
    b = fi.uniform_vector(pb.ndof, seed=22)
    b[dofs] = 0.0
    u_ref = np.linalg.solve(AD, b)
    form = make_form(ctx, case, "elasticity")
    form.set_dirichlet(dofs)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    rc, it, rel = mfa.mfa_cg(ctx.h, form.h, precond, bd, x, 1e-12, 5000)
    assert rc == mfa.MFA_OK and rel <= 1e-12
    u = x.cpu().numpy()
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) <= 1e-9
    assert np.abs(u[dofs]).max() == 0.0


def test_constraint_errors(ctx):
    case = tet_case(2, 2, ncomp=3)
    form = make_form(ctx, case, "elasticity")
    with pytest.raises(mfa.MfaError) as e:
        form.set_dirichlet([0, case["nnode"] * 3])  # one past the last dof
    assert e.value.code == mfa.MFA_ERR_RANGE
    hcase = hex_case(2, 2)
    f64 = make_form(ctx, hcase, "helmholtz")
    f32 = make_form(ctx, hcase, "helmholtz", precision=mfa.MFA_PREC_FP32)
    f32.set_dirichlet([0])
    xf = torch.zeros(hcase["nnode"], dtype=torch.float32, device="cuda")
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_apply_f32(ctx.h, f32.h, xf, torch.empty_like(xf))
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    b = torch.ones(hcase["nnode"], dtype=torch.float64, device="cuda")
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_fcg_mixed(ctx.h, f64.h, f32.h, 4, b, torch.zeros_like(b), 1e-8, 10)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
