"""mfa_cg_noalloc: CG without device allocation, checked against mfa_cg.

Some callers cannot call cudaMalloc (their memory pool already owns the
device memory, or the implicit synchronisation of cudaMalloc/cudaFree would
stall other work in their pipeline).  mfa_cg_noalloc takes its work vectors
from a fixed device array instead.  It must give the same solution as
mfa_cg, call after call, although every call reuses the same array.
"""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import hex_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

# Same bound as the CG tests of the main suite: the solution to within
# 1e-8 of its largest entry.  The Jacobi diagonal is accumulated with f64
# atomics, so two preconditioned solves may differ by rounding that CG
# amplifies; without a preconditioner (and with the coloured scatter) the two
# solvers perform identical arithmetic and must agree bit for bit.
SOL_TOL = 1e-8


def helmholtz_form(ctx, nx, p):
    case = hex_case(nx, p)
    m = mfa.Mesh(ctx, mfa.MFA_CELL_HEX8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, p, 1, case["cell_node"], case["nnode"])
    # coloured scatter: both solvers then do bitwise-identical arithmetic
    # (atomics would add run-to-run rounding that CG amplifies)
    return mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, k2=1.0, scatter=mfa.MFA_SCATTER_COLOUR), case["nnode"]


def solve_both(ctx, form, b, precond):
    bd = torch.from_numpy(b).cuda()
    x_ref = torch.zeros_like(bd)
    rc_ref, it_ref, rel_ref = mfa.mfa_cg(ctx.h, form.h, precond, bd, x_ref, 1e-10, 2000)
    x_new = torch.zeros_like(bd)
    rc_new, it_new, rel_new = mfa.mfa_cg_noalloc(ctx.h, form.h, precond, bd, x_new, 1e-10, 2000)
    assert rc_ref == mfa.MFA_OK and rc_new == mfa.MFA_OK
    assert rel_new <= 1e-10 and rel_ref <= 1e-10
    xr, xn = x_ref.cpu().numpy(), x_new.cpu().numpy()
    assert np.abs(xn - xr).max() <= SOL_TOL * np.abs(xr).max()
    if precond == mfa.MFA_PC_NONE:
        assert it_new == it_ref
        assert np.array_equal(xn.view(np.uint64), xr.view(np.uint64))
    else:
        assert abs(it_new - it_ref) <= 2
    return it_new


def test_noalloc_cg_matches_cg_on_two_calls_in_a_row():
    torch.cuda.set_device(0)
    ctx = mfa.Context(0, torch.cuda.current_stream())
    form1, n1 = helmholtz_form(ctx, 10, 3)  # 29,791 dofs
    form2, n2 = helmholtz_form(ctx, 6, 2)   # 2,197 dofs: a smaller problem after a larger one
    assert n1 <= mfa.MFA_CG_NOALLOC_MAX_NDOF
    it1 = solve_both(ctx, form1, fi.uniform_vector(n1, seed=41), mfa.MFA_PC_JACOBI)
    it2 = solve_both(ctx, form2, fi.uniform_vector(n2, seed=42), mfa.MFA_PC_NONE)
    assert it1 > 0 and it2 > 0


def test_noalloc_cg_allocates_no_device_memory():
    """After a first call (which looks up the array's address), a further call leaves the device's free memory
    unchanged: every work vector comes from the fixed array (cudaMalloc reserves whole 2 MiB pages, so any
    allocation would show)."""
    torch.cuda.set_device(0)
    ctx = mfa.Context(0, torch.cuda.current_stream())
    form, n = helmholtz_form(ctx, 10, 3)
    b = torch.from_numpy(fi.uniform_vector(n, seed=43)).cuda()
    x = torch.zeros_like(b)
    mfa.mfa_cg_noalloc(ctx.h, form.h, mfa.MFA_PC_JACOBI, b, x, 1e-10, 2000)
    x.zero_()
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rc, it, rel = mfa.mfa_cg_noalloc(ctx.h, form.h, mfa.MFA_PC_JACOBI, b, x, 1e-10, 2000)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert rc == mfa.MFA_OK and rel <= 1e-10 and it > 0


def test_noalloc_cg_rejects_sizes_beyond_its_limit():
    torch.cuda.set_device(0)
    ctx = mfa.Context(0, torch.cuda.current_stream())
    form, n = helmholtz_form(ctx, 32, 2)  # 274,625 dofs > 262,144
    assert n > mfa.MFA_CG_NOALLOC_MAX_NDOF
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_cg_noalloc(ctx.h, form.h, mfa.MFA_PC_JACOBI, b, x, 1e-8, 10)
    assert e.value.code == mfa.MFA_ERR_ARG
    assert "limit" in str(e.value)
    assert torch.count_nonzero(x).item() == 0
