"""GPU parity of the FP64 hex vector forms (vector Laplacian, elasticity, SVK and neo-Hookean residual and
Jacobian action) against the FP64 oracle, through the C ABI.  Tolerance 1e-12 relative, as for the scalar forms:
both sides integrate with the same p+1 Gauss points per direction, so they agree to rounding order."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, hex_case, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

TOL = 1e-12
SCATTER = {"atomic": mfa.MFA_SCATTER_ATOMIC, "colour": mfa.MFA_SCATTER_COLOUR}
FORMS = [("laplace", 0), ("elasticity", 0), ("hyper_res", mfa.MFA_LAW_SVK), ("hyper_res", mfa.MFA_LAW_NEOHOOKE),
         ("hyper_jac", mfa.MFA_LAW_SVK), ("hyper_jac", mfa.MFA_LAW_NEOHOOKE)]
NX = {1: 5, 2: 4, 3: 3, 4: 3, 5: 2, 6: 2, 7: 2, 8: 2}  # several blocks, ragged last batch


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], 3, case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def check(y, ref):
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    mx = np.abs(y - ref).max() / np.abs(ref).max()
    assert rel <= TOL and mx <= TOL, (rel, mx)


def inputs(case, kind, seed):
    u = fi.sinusoid_displacement(case["nodes"], seed=seed).ravel()  # smooth, J > 0
    x = fi.uniform_vector(u.size, seed=seed + 50) if kind in ("laplace", "elasticity", "hyper_jac") else u
    return u, x


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kind, law", FORMS)
@pytest.mark.parametrize("scatter", ["atomic", "colour"])
def test_hex_vector_parity(ctx, p, kind, law, scatter):
    case = hex_case(NX[p], p, ncomp=3)
    u, x = inputs(case, kind, seed=p)
    kw = dict(lam=1.3, mu=0.7, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.1, -0.2, 0.05)
    ref = oracle_problem(case, kind, ucoef=u if kind == "hyper_jac" else None, **kw).apply(x)
    form = make_form(ctx, case, kind, scatter=SCATTER[scatter], **kw)
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    check(y.cpu().numpy(), ref)


def test_hex_vector_shuffled_numbering(ctx):
    case = hex_case(3, 3, ncomp=3, shuffle=True)
    u, _ = inputs(case, "hyper_res", seed=9)
    ref = oracle_problem(case, "hyper_res", law=mfa.MFA_LAW_NEOHOOKE).apply(u)
    form = make_form(ctx, case, "hyper_res", law=mfa.MFA_LAW_NEOHOOKE)
    y = form.apply(torch.from_numpy(u).cuda())
    ctx.sync()
    check(y.cpu().numpy(), ref)


def test_hex_vector_colour_is_deterministic(ctx):
    case = hex_case(4, 2, ncomp=3)
    form = make_form(ctx, case, "elasticity", scatter=mfa.MFA_SCATTER_COLOUR)
    x = torch.from_numpy(fi.uniform_vector(case["nnode"] * 3, seed=3)).cuda()
    y1 = form.apply(x).clone()
    y2 = form.apply(x)
    ctx.sync()
    assert torch.equal(y1, y2)


def test_hex_vector_rejections(ctx):
    case = hex_case(2, 2, ncomp=3)
    for kind, kw in [("mass", {}), ("helmholtz", {}), ("elasticity", {"precision": mfa.MFA_PREC_FP32}),
                     ("elasticity", {"qdeg": 5}), ("hyper_res", {"qdeg": 4})]:
        with pytest.raises(mfa.MfaError) as e:
            make_form(ctx, case, kind, **kw)
        assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    form = make_form(ctx, case, "hyper_res")
    with pytest.raises(mfa.MfaError) as e:  # the diagonal covers the linear forms (test_gpu_diag.py)
        form.diagonal()
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    jac = make_form(ctx, case, "hyper_jac")
    with pytest.raises(mfa.MfaError):  # no linearisation point set
        jac.apply(torch.zeros(case["nnode"] * 3, dtype=torch.float64, device="cuda"))


def test_hex_vector_domain_error_is_reported(ctx):
    """A deformation with J <= 0 at a point sets the kernel's error flag (no fault): status MFA_ERR_DOMAIN."""
    case = hex_case(2, 1, ncomp=3)
    form = make_form(ctx, case, "hyper_res", law=mfa.MFA_LAW_NEOHOOKE)
    u = -2.0 * case["nodes"].ravel()  # F = -I: det F = -1
    form.apply(torch.from_numpy(u).cuda())
    with pytest.raises(mfa.MfaError) as e:
        ctx.sync()
    assert e.value.code == mfa.MFA_ERR_DOMAIN


@pytest.mark.parametrize("p, kind, law", [(1, "elasticity", 0), (3, "elasticity", 0), (6, "elasticity", 0),
                                          (2, "laplace", 0), (1, "hyper_res", mfa.MFA_LAW_NEOHOOKE),
                                          (2, "hyper_jac", mfa.MFA_LAW_SVK), (3, "hyper_res", mfa.MFA_LAW_SVK),
                                          (3, "hyper_jac", mfa.MFA_LAW_NEOHOOKE)])
def test_hex_vector_table2_quadrature(ctx, p, kind, law):
    """Table 2's rules on hexahedra: p+2 points per direction for the linear vector forms, 2p+2 for
    hyperelasticity."""
    qdeg = 2 * p + 2 if kind.startswith("hyper") else p + 2
    case = hex_case({1: 4, 2: 3, 3: 2, 6: 2}[p], p, ncomp=3)
    u, x = inputs(case, kind, seed=20 + p)
    kw = dict(lam=1.1, mu=0.9, law=law)
    ref = oracle_problem(case, kind, qdeg=qdeg, ucoef=u if kind == "hyper_jac" else None, **kw).apply(x)
    form = make_form(ctx, case, kind, qdeg=qdeg, **kw)
    assert form.info().nq == qdeg ** 3
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    check(y.cpu().numpy(), ref)
