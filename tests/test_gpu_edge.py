"""Edge cases on every kernel family: an empty mesh gives y = 0 without error, and a flat mesh (every cell's
Jacobian determinant zero) is reported as MFA_ERR_DOMAIN, at form creation where the geometric factors are
stored, else at the next synchronisation, without a fault; the context stays usable afterwards."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, hex_case, oracle_problem, quad_case, tet_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

# (label, case builder, form, form keywords): one per kernel family
FAMILIES = [
    ("hex-point-Q2", lambda: hex_case(2, 2), "helmholtz", {}),
    ("hex-even-odd-Q6", lambda: hex_case(1, 6), "laplace", {}),
    ("hex-fp32-line-Q3", lambda: hex_case(2, 3), "helmholtz", {"precision": mfa.MFA_PREC_FP32}),
    ("hex-vector-Q2", lambda: hex_case(2, 2, ncomp=3), "elasticity", {}),
    ("tet-P1", lambda: tet_case(2, 1), "mass", {}),
    ("tet-P2-vector", lambda: tet_case(2, 2, ncomp=3), "elasticity", {}),
    ("tet-P2-moment", lambda: tet_case(2, 2, ncomp=3), "hyper_res", {"law": mfa.MFA_LAW_SVK}),
    ("tet-P3-dense", lambda: tet_case(1, 3), "helmholtz", {}),
    ("tri-P2-cell", lambda: tri_case(3, 2), "helmholtz", {}),
    ("tri-P5-dense", lambda: tri_case(2, 5), "laplace", {}),
    ("quad-Q3", lambda: quad_case(3, 3), "helmholtz", {}),
]


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def ndof(case):
    return case["nnode"] * case["ncomp"]


@pytest.mark.parametrize("label, builder, kind, kw", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_empty_mesh(ctx, label, builder, kind, kw):
    case = builder()
    case["cell_vert"] = case["cell_vert"][:0]
    case["cell_node"] = case["cell_node"][:0]
    form = make(ctx, case, kind, **kw)
    x = torch.ones(ndof(case), dtype=torch.float64, device="cuda")
    y = torch.full_like(x, np.nan)
    mfa.mfa_apply(ctx.h, form.h, x, y)
    ctx.sync()
    assert torch.all(y == 0)


@pytest.mark.parametrize("label, builder, kind, kw", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_flat_mesh_reports_domain_error(ctx, label, builder, kind, kw):
    case = builder()
    flat = dict(case)
    coords = np.array(case["coords"], dtype=np.float64)
    coords[:, 0] = 0.0  # every cell collapses onto the plane x = 0 (onto a line in the plane)
    flat["coords"] = coords
    x = torch.from_numpy(fi.uniform_vector(ndof(case), seed=3)).cuda()
    with pytest.raises(mfa.MfaError) as e:
        form = make(ctx, flat, kind, **kw)
        form.apply(x)
        ctx.sync()
    assert e.value.code == mfa.MFA_ERR_DOMAIN
    # the flag was cleared and the context still works: the same form on the undeformed mesh matches the oracle
    good = make(ctx, case, kind, **kw)
    y = good.apply(x)
    ctx.sync()
    okw = {k: v for k, v in kw.items() if k != "precision"}
    ref = oracle_problem(case, kind, **okw).apply(x.cpu().numpy())
    tol = 1e-5 if "precision" in kw else 1e-12
    assert np.linalg.norm(y.cpu().numpy() - ref) <= tol * np.linalg.norm(ref)
