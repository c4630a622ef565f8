"""The building blocks of the overlapped distributed apply on the GPU: for each rank's cells (the halo plan of
paper_1903_08243_gb300.dist), a form over the boundary cells applied first and a form over the interior cells
applied with accumulate give the action of one form over all the rank's cells, and match the oracle."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, hex_case, oracle_problem, tet_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402
from paper_1903_08243_gb300 import dist as mdist  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def local_form(ctx, case, plan, sel, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"][plan.cells[sel]])
    sp = mfa.Space(m, case["degree"], case["ncomp"], np.ascontiguousarray(plan.local_cell_node[sel]), plan.l2g.size)
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


@pytest.mark.parametrize("which", ["hex-Q3-helmholtz", "tet-P2-elasticity"])
@pytest.mark.parametrize("nranks", [2, 3])
def test_boundary_then_interior_equals_whole_rank(ctx, which, nranks):
    if which.startswith("hex"):
        case, kind, kw = hex_case(9, 3), "helmholtz", {"k2": 0.8}  # 9 layers: every rank keeps interior cells
    else:
        case, kind, kw = tet_case(9, 2, ncomp=3, perturb=0.1, seed=5), "elasticity", {"lam": 1.2, "mu": 0.7}
    nc = case["ncomp"]
    x = fi.uniform_vector(case["nnode"] * nc, seed=11).reshape(-1, nc)
    for rank in range(nranks):
        plan = mdist.build_plan(case["cell_node"], case["nnode"], nranks, rank)
        assert len(plan.interior_cells) > 0 and len(plan.boundary_cells) > 0
        whole = local_form(ctx, case, plan, np.arange(len(plan.cells)), kind, **kw)
        fb = local_form(ctx, case, plan, plan.boundary_cells, kind, **kw)
        fi_ = local_form(ctx, case, plan, plan.interior_cells, kind, **kw)
        xl = torch.from_numpy(np.ascontiguousarray(x[plan.l2g]).reshape(-1)).cuda()
        y_whole = whole.apply(xl)
        y = torch.empty_like(xl)
        mfa.mfa_apply(ctx.h, fb.h, xl, y, False)
        mfa.mfa_apply(ctx.h, fi_.h, xl, y, True)
        ctx.sync()
        a, b = y.cpu().numpy(), y_whole.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)
        # and the rank's part of the global action: the oracle over the rank's cells in its local numbering
        ref = oracle_problem(dict(case, cell_vert=case["cell_vert"][plan.cells], cell_node=plan.local_cell_node,
                                  nnode=plan.l2g.size), kind, **kw).apply(xl.cpu().numpy())
        assert np.linalg.norm(a - ref) <= 1e-12 * np.linalg.norm(ref)
