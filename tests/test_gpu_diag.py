"""mfa_diagonal on every cell type against the diagonal assembled from the oracle's element matrices: quadrilaterals, triangles,
tetrahedra P3-P5 and the hex vector forms (scalar hex and P1/P2 tets are covered in test_gpu_parity.py), and
Jacobi-PCG on a planar and a P3 tet problem."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, assembled_dense, hex_case, oracle_problem, quad_case, tet_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

CASES = [
    ("quad-Q1-mass", lambda: quad_case(4, 1), "mass", {}, {}),
    ("quad-Q3-laplace", lambda: quad_case(3, 3), "laplace", {}, {}),
    ("quad-Q3-helmholtz", lambda: quad_case(3, 3), "helmholtz", {"k2": 0.7}, {}),
    ("quad-Q2-helmholtz-p+2", lambda: quad_case(3, 2), "helmholtz", {"k2": 0.7}, {"qdeg": 4}),
    ("quad-Q2-elasticity", lambda: quad_case(3, 2, ncomp=2), "elasticity", {"lam": 1.3, "mu": 0.6}, {}),
    ("quad-Q2-vector-laplace", lambda: quad_case(3, 2, ncomp=2), "laplace", {}, {}),
    ("tri-P1-helmholtz", lambda: tri_case(4, 1), "helmholtz", {"k2": 0.9}, {}),
    ("tri-P2-mass", lambda: tri_case(3, 2), "mass", {}, {}),
    ("tri-P3-laplace", lambda: tri_case(3, 3), "laplace", {}, {}),
    ("tri-P5-helmholtz", lambda: tri_case(2, 5), "helmholtz", {"k2": 0.9}, {}),
    ("tri-P2-elasticity", lambda: tri_case(3, 2, ncomp=2), "elasticity", {"lam": 1.3, "mu": 0.6}, {}),
    ("tri-P4-elasticity", lambda: tri_case(2, 4, ncomp=2), "elasticity", {"lam": 1.3, "mu": 0.6}, {}),
    ("tet-P3-helmholtz", lambda: tet_case(2, 3, perturb=0.1, seed=3), "helmholtz", {"k2": 0.9}, {}),
    ("tet-P4-laplace", lambda: tet_case(1, 4, perturb=0.1, seed=3), "laplace", {}, {}),
    ("tet-P5-mass", lambda: tet_case(1, 5, perturb=0.1, seed=3), "mass", {}, {}),
    ("tet-P3-elasticity", lambda: tet_case(1, 3, ncomp=3, perturb=0.1, seed=3), "elasticity",
     {"lam": 1.3, "mu": 0.6}, {}),
    ("hex-vector-Q2-elasticity", lambda: hex_case(2, 2, ncomp=3), "elasticity", {"lam": 1.3, "mu": 0.6}, {}),
    ("hex-vector-Q2-laplace", lambda: hex_case(2, 2, ncomp=3), "laplace", {}, {}),
    ("hex-vector-Q1-elasticity-p+2", lambda: hex_case(3, 1, ncomp=3), "elasticity", {"lam": 1.3, "mu": 0.6},
     {"qdeg": 3}),
]


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def oracle_diagonal(pb, case):
    """Diagonal assembled from the oracle's element matrices (local dofs a * ncomp + c)."""
    nc, cn = case["ncomp"], case["cell_node"]
    d = np.zeros(case["nnode"] * nc)
    for cell in range(cn.shape[0]):
        de = np.diag(pb.element_matrix(cell))
        for a in range(cn.shape[1]):
            for c in range(nc):
                d[nc * cn[cell, a] + c] += de[a * nc + c]
    return d


@pytest.mark.parametrize("label, builder, kind, kw, rule", CASES, ids=[c[0] for c in CASES])
def test_diagonal_matches_dense_oracle(ctx, label, builder, kind, kw, rule):
    case = builder()
    ref = oracle_diagonal(oracle_problem(case, kind, qdeg=rule.get("qdeg"), **kw), case)
    form = make(ctx, case, kind, qdeg=rule.get("qdeg", 0), **kw)
    d = form.diagonal()
    ctx.sync()
    d = d.cpu().numpy()
    assert np.linalg.norm(d - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.abs(d - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("which", ["quad-Q3", "tri-P4", "tet-P3"])
def test_jacobi_pcg(ctx, which):
    case = {"quad-Q3": lambda: quad_case(5, 3), "tri-P4": lambda: tri_case(5, 4),
            "tet-P3": lambda: tet_case(2, 3, perturb=0.1, seed=3)}[which]()
    kw = {"k2": 1.0}
    A = assembled_dense(oracle_problem(case, "helmholtz", **kw), case)
    b = fi.uniform_vector(case["nnode"], seed=12)
    xs = np.linalg.solve(A, b)
    form = make(ctx, case, "helmholtz", **kw)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    rc, it, rel = form.cg(bd, xd, precond=mfa.MFA_PC_JACOBI, rtol=1e-12, maxit=2000)
    assert rc == mfa.MFA_OK and rel <= 1e-12
    np.testing.assert_allclose(xd.cpu().numpy(), xs, rtol=0, atol=1e-8 * np.abs(xs).max())


def test_diagonal_limits(ctx):
    case = tet_case(1, 2, ncomp=3)
    f = make(ctx, case, "hyper_res", law=mfa.MFA_LAW_SVK)
    with pytest.raises(mfa.MfaError) as e:
        f.diagonal()
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
