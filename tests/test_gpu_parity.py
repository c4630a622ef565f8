"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance (FP64 paths): relative L2 error <= 1e-12 and max-abs error <= 1e-12
times max|y_ref|.  Both sides integrate the same forms with rules that are
exact for the polynomial integrands (or the same conical-product rule for
neo-Hookean), so they agree to rounding; reordering of FP64 sums over
~10^2-10^3 terms per entry stays many orders below the bound.
"""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
from tests.problems import KIND_NAMES, cells_touching, hex_case, oracle_problem, quad_case, tet_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

TOL = 1e-12
SCATTER = {"atomic": mfa.MFA_SCATTER_ATOMIC, "colour": mfa.MFA_SCATTER_COLOUR}
LAWS = {"svk": mfa.MFA_LAW_SVK, "nh": mfa.MFA_LAW_NEOHOOKE}


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    c = mfa.Context(0, torch.cuda.current_stream())
    yield c


def gpu_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def compare(y, ref, tol=TOL):
    y = np.asarray(y)
    rel = np.linalg.norm(y - ref) / max(np.linalg.norm(ref), 1e-300)
    mx = np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert rel <= tol and mx <= tol, (rel, mx)
    return rel


def run(ctx, form, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = form.apply(xd)
    ctx.sync()
    return y.cpu().numpy()


# ------------------------------------------------------------------ hexahedra

@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("scatter", ["atomic", "colour"])
def test_hex_parity(ctx, p, kind, scatter):
    nx = {1: 7, 2: 5, 3: 5, 4: 3, 5: 3, 6: 3, 7: 2, 8: 2}[p]  # several blocks and a ragged last batch
    case = hex_case(nx, p)
    x = fi.uniform_vector(case["nnode"], seed=11)
    ref = oracle_problem(case, kind, k2=0.75).apply(x)
    form = gpu_form(ctx, case, kind, k2=0.75, scatter=SCATTER[scatter])
    compare(run(ctx, form, x), ref)


PREC = {"fp32": (mfa.MFA_PREC_FP32, 1e-5), "bf16": (mfa.MFA_PREC_BF16, 1e-2)}


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_hex_mixed_precision_against_fp64_oracle(ctx, p, kind, prec):
    """FP32 arithmetic within 1e-5, BF16 operands with FP32 accumulation within 1e-2 (relative L2)."""
    nx = {1: 7, 2: 5, 3: 5, 4: 3, 5: 3, 6: 3, 7: 2, 8: 2}[p]
    case = hex_case(nx, p)
    x = fi.uniform_vector(case["nnode"], seed=16)
    ref = oracle_problem(case, kind, k2=1.0).apply(x)
    code, tol = PREC[prec]
    form = gpu_form(ctx, case, kind, k2=1.0, precision=code)
    y = run(ctx, form, x)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel <= tol, rel
    if prec == "fp32":
        assert rel > 1e-12  # really computed in reduced precision


@pytest.mark.parametrize("p", [1, 4, 8])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_apply_f32_vectors(ctx, p, prec):
    nx = {1: 7, 4: 3, 8: 2}[p]
    case = hex_case(nx, p)
    x = fi.uniform_vector(case["nnode"], seed=17)
    ref = oracle_problem(case, "helmholtz").apply(x)
    code, tol = PREC[prec]
    form = gpu_form(ctx, case, "helmholtz", precision=code)
    xf = torch.from_numpy(x).cuda().float()
    yf = torch.empty_like(xf)
    mfa.mfa_apply_f32(ctx.h, form.h, xf, yf)
    ctx.sync()
    y = yf.double().cpu().numpy()
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= tol
    # same result as the double-vector entry point up to the float rounding of the output
    yd = run(ctx, form, x)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) <= 1e-6


def test_integer_pipe_conversions_match_cuda(ctx):
    rng = np.random.default_rng(3)
    mant = rng.standard_normal(200000)
    expo = rng.integers(-120, 120, size=mant.size)
    x = np.ldexp(mant, expo)
    x[:8] = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 3.4028234663852886e38, 1.1754943508222875e-38]
    # ties: exactly halfway between two floats, both parities
    halfway = np.array([1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -(2.0 + 2.0 ** -23)])
    x = np.concatenate([x, halfway])
    xd = torch.from_numpy(x).cuda()
    yf = torch.empty(x.size, dtype=torch.float32, device="cuda")
    mfa.mfa_convert_f64_to_f32(ctx.h, xd, yf)
    ctx.sync()
    ref = xd.float()  # CUDA's own round-to-nearest conversion
    normal = torch.isfinite(ref) & ((ref.abs() >= 1.1754943508222875e-38) | (ref == 0))
    assert torch.equal(yf[normal].view(torch.int32), ref[normal].view(torch.int32))
    assert torch.equal(torch.isinf(yf), torch.isinf(ref))
    back = torch.empty_like(xd)
    mfa.mfa_convert_f32_to_f64(ctx.h, yf, back)
    ctx.sync()
    fin = torch.isfinite(yf) & ((yf.abs() >= 1.1754943508222875e-38) | (yf == 0))
    assert torch.equal(back[fin].view(torch.int64), yf[fin].double().view(torch.int64))


def test_mixed_precision_rejected_where_not_built(ctx):
    case = tet_case(2, 1)
    with pytest.raises(mfa.MfaError) as e:
        gpu_form(ctx, case, "mass", precision=mfa.MFA_PREC_FP32)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED


@pytest.mark.parametrize("p", [1, 3, 6])
def test_hex_paper_quadrature_p_plus_2(ctx, p):
    """Table 2 uses p+2 Gauss points per direction on hexahedra."""
    case = hex_case(3, p)
    x = fi.uniform_vector(case["nnode"], seed=12)
    ref = oracle_problem(case, "helmholtz", qdeg=p + 2).apply(x)
    form = gpu_form(ctx, case, "helmholtz", qdeg=p + 2)
    compare(run(ctx, form, x), ref)


def test_hex_shuffled_numbering(ctx):
    case = hex_case(4, 3, shuffle=True)
    x = fi.uniform_vector(case["nnode"], seed=13)
    ref = oracle_problem(case, "laplace").apply(x)
    for sc in SCATTER.values():
        compare(run(ctx, gpu_form(ctx, case, "laplace", scatter=sc), x), ref)


def test_colour_scatter_is_bitwise_deterministic(ctx):
    case = hex_case(6, 3)
    x = fi.uniform_vector(case["nnode"], seed=14)
    form = gpu_form(ctx, case, "helmholtz", scatter=mfa.MFA_SCATTER_COLOUR)
    assert form.info().ncolours == 8
    y1, y2 = run(ctx, form, x), run(ctx, form, x)
    assert np.array_equal(y1.view(np.uint64), y2.view(np.uint64))


def test_hex_accumulate_and_host_apply(ctx):
    case = hex_case(4, 2)
    x = fi.uniform_vector(case["nnode"], seed=15)
    ref = oracle_problem(case, "mass").apply(x)
    form = gpu_form(ctx, case, "mass")
    compare(form.apply_host(x), ref)
    xd = torch.from_numpy(x).cuda()
    y = torch.ones_like(xd)
    form.apply(xd, y, accumulate=True)
    ctx.sync()
    compare(y.cpu().numpy(), ref + 1.0)


@pytest.mark.parametrize("p", [1, 4])
def test_hex_full_size_sampled(ctx, p):
    """64^3 perturbed hex mesh (the benchmark size): sampled dofs against the oracle, cell by cell."""
    case = hex_case(64, p)
    x = fi.uniform_vector(case["nnode"], seed=1)
    form = gpu_form(ctx, case, "helmholtz")
    y = run(ctx, form, x)
    rng = np.random.default_rng(p)
    dofs = rng.choice(case["nnode"], size=64, replace=False)
    cells = cells_touching(case["cell_node"], dofs)
    ref = oracle_problem(case, "helmholtz").apply(x, cells=cells)
    compare(y[dofs], ref[dofs])
    # the action of the constant field sums to the domain volume (k2 = 1)
    one = run(ctx, form, np.ones(case["nnode"]))
    assert abs(one.sum() - 1.0) < 1e-11


def test_empty_mesh(ctx):
    case = hex_case(2, 2)
    case["cell_vert"] = case["cell_vert"][:0]
    case["cell_node"] = case["cell_node"][:0]
    form = gpu_form(ctx, case, "helmholtz")
    y = run(ctx, form, np.ones(case["nnode"]))
    assert np.all(y == 0)


# ------------------------------------------------------------------ tetrahedra

TET_CASES = [
    (1, 1, "mass", {}), (1, 1, "laplace", {}), (1, 1, "helmholtz", {"k2": 0.5}),
    (2, 1, "mass", {}), (2, 1, "laplace", {}), (2, 1, "helmholtz", {"k2": 2.0}),
    (2, 3, "laplace", {}), (2, 3, "elasticity", {"lam": 1.0, "mu": 1.0}),
    (2, 3, "elasticity", {"lam": 0.0, "mu": 0.5}),  # the paper's int eps(u):eps(v)
]


@pytest.mark.parametrize("p,ncomp,kind,kw", TET_CASES)
@pytest.mark.parametrize("scatter", ["atomic", "colour"])
def test_tet_linear_forms(ctx, p, ncomp, kind, kw, scatter):
    case = tet_case(5, p, ncomp=ncomp, perturb=0.15, seed=3)
    x = fi.uniform_vector(case["nnode"] * ncomp, seed=21)
    ref = oracle_problem(case, kind, **kw).apply(x)
    form = gpu_form(ctx, case, kind, scatter=SCATTER[scatter], **kw)
    compare(run(ctx, form, x), ref)


@pytest.mark.parametrize("law", ["svk", "nh"])
@pytest.mark.parametrize("scatter", ["atomic", "colour"])
def test_tet_hyperelastic_residual(ctx, law, scatter):
    case = tet_case(4, 2, ncomp=3, perturb=0.15, seed=4)
    u = fi.sinusoid_displacement(case["nodes"], seed=2).ravel()
    b = (0.1, -0.2, 0.05)
    ref = oracle_problem(case, "hyper_res", law=LAWS[law], b=b).apply(u)
    form = gpu_form(ctx, case, "hyper_res", law=LAWS[law], b=b, scatter=SCATTER[scatter])
    compare(run(ctx, form, u), ref)


@pytest.mark.parametrize("law", ["svk", "nh"])
def test_tet_hyperelastic_jacobian(ctx, law):
    case = tet_case(4, 2, ncomp=3, perturb=0.15, seed=5)
    u = fi.sinusoid_displacement(case["nodes"], seed=3).ravel()
    du = fi.uniform_vector(u.size, seed=22)
    ref = oracle_problem(case, "hyper_jac", law=LAWS[law], ucoef=u).apply(du)
    form = gpu_form(ctx, case, "hyper_jac", law=LAWS[law])
    ud = torch.from_numpy(u).cuda()
    form.set_coefficient(ud)
    compare(run(ctx, form, du), ref)


def test_tet_p1_mass_config0_full(ctx):
    """The 8^3 x 6 Kuhn mesh, P1 mass, in full."""
    case = tet_case(8, 1)
    x = fi.uniform_vector(case["nnode"], seed=0)
    ref = oracle_problem(case, "mass").apply(x)
    for sc in SCATTER.values():
        compare(run(ctx, gpu_form(ctx, case, "mass", scatter=sc), x), ref)


def test_tet_p2_elasticity_and_nh_full_size_sampled(ctx):
    """48^3 x 6 Kuhn mesh, vector P2: sampled dofs against the oracle, cell by cell."""
    case = tet_case(48, 2, ncomp=3)
    u = fi.sinusoid_displacement(case["nodes"], seed=2).ravel()
    rng = np.random.default_rng(9)
    dofs = rng.choice(u.size, size=48, replace=False)
    cells = cells_touching(case["cell_node"], dofs, ncomp=3)
    for kind, kw in [("elasticity", {}), ("hyper_res", {"law": mfa.MFA_LAW_NEOHOOKE})]:
        okw = {"law": oracle.NEOHOOKE} if kw else {}
        y = run(ctx, gpu_form(ctx, case, kind, **kw), u)
        ref = oracle_problem(case, kind, **okw).apply(u, cells=cells)
        compare(y[dofs], ref[dofs])


def test_tet_shuffled(ctx):
    case = tet_case(4, 2, ncomp=3, perturb=0.1, seed=6, shuffle=True)
    x = fi.uniform_vector(case["nnode"] * 3, seed=23)
    ref = oracle_problem(case, "elasticity").apply(x)
    compare(run(ctx, gpu_form(ctx, case, "elasticity"), x), ref)


# ------------------------------------------------------------------ diagonal and CG

@pytest.mark.parametrize("which", ["hex-helm", "hex-lap", "hex-mass", "tet-p1-helm", "tet-p2-elast"])
def test_diagonal(ctx, which):
    if which.startswith("hex"):
        case = hex_case(2, 3)
        kind = {"helm": "helmholtz", "lap": "laplace", "mass": "mass"}[which.split("-")[1]]
        kw = {"k2": 0.6} if kind == "helmholtz" else {}
    elif which == "tet-p1-helm":
        case, kind, kw = tet_case(2, 1, perturb=0.2, seed=7), "helmholtz", {"k2": 0.6}
    else:
        case, kind, kw = tet_case(2, 2, ncomp=3, perturb=0.2, seed=7), "elasticity", {"lam": 1.3, "mu": 0.7}
    ref = np.diag(oracle_problem(case, kind, **kw).dense())
    form = gpu_form(ctx, case, kind, **kw)
    d = form.diagonal()
    ctx.sync()
    compare(d.cpu().numpy(), ref)


@pytest.mark.parametrize("precond", [mfa.MFA_PC_NONE, mfa.MFA_PC_JACOBI])
def test_cg_matches_dense_solve(ctx, precond):
    case = hex_case(3, 2)
    A = oracle_problem(case, "helmholtz").dense()
    b = fi.uniform_vector(case["nnode"], seed=30)
    xs = np.linalg.solve(A, b)
    form = gpu_form(ctx, case, "helmholtz")
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    rc, it, rel = form.cg(bd, xd, precond=precond, rtol=1e-12, maxit=500)
    assert rc == mfa.MFA_OK and rel <= 1e-12
    # The error is bounded by the residual: ||x - x*|| / ||x*|| <= kappa_2(A) ||b - A x|| / ||b||.  This matrix has
    # kappa_2 ~ 605, so a residual of 1e-12 allows a relative error of ~6e-10 in the 2-norm (~4e-9 of max|x*| in
    # the max-norm here, which is why a max-norm bound of 1e-9 max|x*| does not follow).  The residual is taken
    # again on the host with the dense matrix; 1e-13 covers the rounding of the dense solve itself (kappa eps).
    x = xd.cpu().numpy()
    ev = np.linalg.eigvalsh(A)
    kappa = ev.max() / ev.min()
    true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert true_rel <= 2e-12
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * true_rel + 1e-13, (kappa, true_rel)


@pytest.mark.parametrize("precond", [mfa.MFA_PC_NONE, mfa.MFA_PC_JACOBI])
def test_cg_error_decreases_in_the_energy_norm(ctx, precond):
    """(P)CG minimises the A-norm of the error over a growing Krylov space, so from x0 = 0 the iterate after k
    steps is at least as close to the solution in that norm as the iterate after k - 1 (dense oracle matrix)."""
    case = hex_case(3, 2)
    A = oracle_problem(case, "helmholtz", k2=0.5).dense()
    b = fi.uniform_vector(case["nnode"], seed=31)
    xs = np.linalg.solve(A, b)
    form = gpu_form(ctx, case, "helmholtz", k2=0.5)
    bd = torch.from_numpy(b).cuda()
    errs = []
    for k in range(1, 16):
        xd = torch.zeros_like(bd)
        rc, it, rel = form.cg(bd, xd, precond=precond, rtol=1e-30, maxit=k)
        assert rc == mfa.MFA_ERR_NOT_CONVERGED and it == k
        e = xd.cpu().numpy() - xs
        errs.append(float(np.sqrt(e @ A @ e)))
    e0 = float(np.sqrt(xs @ A @ xs))
    assert errs[0] < e0
    for k in range(1, len(errs)):
        assert errs[k] <= errs[k - 1] * (1 + 1e-12), (k, errs[k - 1], errs[k])
    assert errs[-1] < 0.5 * errs[0]


@pytest.mark.parametrize("inner_prec,inner_iters", [("fp64", 0), ("fp32", 6), ("bf16", 4), ("fp64", 10)])
def test_fcg_mixed_matches_dense_solve(ctx, inner_prec, inner_iters):
    case = hex_case(4, 2)
    A = oracle_problem(case, "helmholtz").dense()
    b = fi.uniform_vector(case["nnode"], seed=32)
    xs = np.linalg.solve(A, b)
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, 2, 1, case["cell_node"], case["nnode"])
    outer = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    code = {"fp64": mfa.MFA_PREC_FP64, "fp32": mfa.MFA_PREC_FP32, "bf16": mfa.MFA_PREC_BF16}[inner_prec]
    inner = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, precision=code)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    rc, it, inn, rel = mfa.mfa_fcg_mixed(ctx.h, outer.h, inner.h, inner_iters, bd, xd, 1e-11, 400)
    assert rc == mfa.MFA_OK and rel <= 1e-11
    x = xd.cpu().numpy()
    assert np.linalg.norm(b - A @ x) <= 2e-11 * np.linalg.norm(b)  # the FP64 residual, recomputed
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-8 * np.abs(xs).max())
    if inner_iters:
        rc0, it0, _, _ = mfa.mfa_fcg_mixed(ctx.h, outer.h, inner.h, 0, bd, torch.zeros_like(bd), 1e-11, 400)
        assert it < it0  # the inner solve cuts outer iterations


def test_cg_not_converged_status(ctx):
    case = hex_case(3, 2)
    form = gpu_form(ctx, case, "helmholtz")
    bd = torch.from_numpy(fi.uniform_vector(case["nnode"], seed=31)).cuda()
    rc, it, rel = form.cg(bd, torch.zeros_like(bd), precond=mfa.MFA_PC_NONE, rtol=1e-14, maxit=3)
    assert rc == mfa.MFA_ERR_NOT_CONVERGED and it == 3


def test_cg_breakdown_on_nan(ctx):
    case = hex_case(2, 1)
    form = gpu_form(ctx, case, "helmholtz")
    b = np.ones(case["nnode"])
    b[3] = np.nan
    bd = torch.from_numpy(b).cuda()
    with pytest.raises(mfa.MfaError) as e:
        form.cg(bd, torch.zeros_like(bd), rtol=1e-8, maxit=10)
    assert e.value.code == mfa.MFA_ERR_BREAKDOWN


# ------------------------------------------------------------------ errors found on the host or by kernels

def test_range_errors(ctx):
    case = hex_case(2, 1)
    bad = case["cell_vert"].copy()
    bad[1, 3] = case["coords"].shape[0]
    with pytest.raises(mfa.MfaError) as e:
        mfa.Mesh(ctx, 8, case["coords"], bad)
    assert e.value.code == mfa.MFA_ERR_RANGE
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    cn = case["cell_node"].copy()
    cn[0, 0] = -1
    with pytest.raises(mfa.MfaError) as e:
        mfa.Space(m, 1, 1, cn, case["nnode"])
    assert e.value.code == mfa.MFA_ERR_RANGE
    cn = case["cell_node"].copy()
    cn[0, 1] = cn[0, 0]
    with pytest.raises(mfa.MfaError) as e:
        mfa.Space(m, 1, 1, cn, case["nnode"])
    assert e.value.code == mfa.MFA_ERR_ARG


def test_unsupported_combinations(ctx):
    case = hex_case(2, 1)
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, 1, 1, case["cell_node"], case["nnode"])
    with pytest.raises(mfa.MfaError) as e:
        mfa.Form(sp, mfa.MFA_FORM_ELASTICITY)
    assert e.value.code == mfa.MFA_ERR_ARG
    with pytest.raises(mfa.MfaError) as e:
        mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, qdeg=7)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED


def test_neohookean_inverted_element_reports_domain_error(ctx):
    case = tet_case(2, 2, ncomp=3)
    u = -3.0 * case["nodes"].ravel()  # F = -2 I: det F < 0 everywhere
    form = gpu_form(ctx, case, "hyper_res", law=mfa.MFA_LAW_NEOHOOKE)
    form.apply(torch.from_numpy(u).cuda())
    with pytest.raises(mfa.MfaError) as e:
        ctx.sync()
    assert e.value.code == mfa.MFA_ERR_DOMAIN
    ctx.sync()  # the flag was cleared


# ------------------------------------------------------------------ batched operators

def _batch_inputs(ctx):
    rng = np.random.default_rng(77)
    forms, xs, refs = [], [], []
    specs = [(1, "helmholtz", "fp64"), (2, "laplace", "fp64"), (2, "laplace", "fp64"), (3, "mass", "fp32"),
             (3, "helmholtz", "fp32"), (4, "helmholtz", "bf16"), (2, "helmholtz", "fp32"), (8, "helmholtz", "fp64"),
             (5, "helmholtz", "fp64")]
    keep = []
    for i, (p, kind, prec) in enumerate(specs):
        nx = int(rng.integers(2, 5))
        case = hex_case(nx, p, seed=100 + i)
        code = {"fp64": mfa.MFA_PREC_FP64, "fp32": mfa.MFA_PREC_FP32, "bf16": mfa.MFA_PREC_BF16}[prec]
        f = gpu_form(ctx, case, kind, k2=1.0, precision=code)
        x = fi.uniform_vector(case["nnode"], seed=200 + i)
        forms.append(f)
        xs.append(torch.from_numpy(x).cuda())
        refs.append((oracle_problem(case, kind, k2=1.0).apply(x), {"fp64": 1e-12, "fp32": 1e-5, "bf16": 1e-2}[prec]))
        keep.append(case)
    # two forms that cannot be grouped: a tetrahedral one and a coloured one
    tcase = tet_case(3, 2, ncomp=3, perturb=0.1, seed=9)
    f = gpu_form(ctx, tcase, "elasticity")
    x = fi.uniform_vector(tcase["nnode"] * 3, seed=300)
    forms.append(f)
    xs.append(torch.from_numpy(x).cuda())
    refs.append((oracle_problem(tcase, "elasticity").apply(x), 1e-12))
    hcase = hex_case(3, 2, seed=5)
    f = gpu_form(ctx, hcase, "helmholtz", scatter=mfa.MFA_SCATTER_COLOUR)
    x = fi.uniform_vector(hcase["nnode"], seed=301)
    forms.append(f)
    xs.append(torch.from_numpy(x).cuda())
    refs.append((oracle_problem(hcase, "helmholtz").apply(x), 1e-12))
    # and two planar ones (a quad and a triangle form)
    for pcase, kind, seed in [(quad_case(4, 3), "helmholtz", 302), (tri_case(4, 2, ncomp=2), "elasticity", 303)]:
        f = gpu_form(ctx, pcase, kind)
        x = fi.uniform_vector(pcase["nnode"] * pcase["ncomp"], seed=seed)
        forms.append(f)
        xs.append(torch.from_numpy(x).cuda())
        refs.append((oracle_problem(pcase, kind).apply(x), 1e-12))
    return forms, xs, refs


def _check_batch(ys, refs):
    for y, (ref, tol) in zip(ys, refs):
        yv = y.cpu().numpy()
        rel = np.linalg.norm(yv - ref) / np.linalg.norm(ref)
        assert rel <= tol, (rel, tol)


def test_apply_batched(ctx):
    forms, xs, refs = _batch_inputs(ctx)
    ys = [torch.full_like(x, 7.0) for x in xs]  # overwritten, not accumulated
    mfa.mfa_apply_batched(ctx.h, [f.h for f in forms], xs, ys)
    _check_batch(ys, refs)


def test_batch_graph_replay(ctx):
    forms, xs, refs = _batch_inputs(ctx)
    ys = [torch.empty_like(x) for x in xs]
    b = mfa.mfa_batch_create(ctx.h, [f.h for f in forms], xs, ys)
    try:
        ngroups, nsingles = mfa.mfa_batch_info(b)
        # (1,H,64) (2,L,64) (3,M,32) (3,H,32) (4,H,16) (2,H,32) (8,H,64) (5,H,64: the even-odd group kernel)
        assert nsingles == 4 and ngroups == 8
        for y in ys:
            y.fill_(-1.0)
        for _ in range(2):
            mfa.mfa_batch_apply(ctx.h, b)
        ctx.sync()
        _check_batch(ys, refs)
    finally:
        mfa.mfa_batch_destroy(b)


def test_handles_may_be_destroyed_after_their_context(ctx):
    """Python's collector may finalise a context before the forms built on it (reference cycles through
    tracebacks); destroying the form afterwards must neither touch the freed context nor leave an error
    behind for the next launch."""
    case = hex_case(2, 2)
    c2 = mfa.Context(0, torch.cuda.current_stream())
    m = mfa.Mesh(c2, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, 2, 1, case["cell_node"], case["nnode"])
    f = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    hf, hs, hm = f.h, sp.h, m.h
    f.h = sp.h = m.h = None  # destroy by hand, context first
    c2.close()
    mfa.mfa_form_destroy(hf)
    mfa.mfa_space_destroy(hs)
    mfa.mfa_mesh_destroy(hm)
    x = fi.uniform_vector(case["nnode"], seed=30)
    ref = oracle_problem(case, "helmholtz").apply(x)
    compare(run(ctx, gpu_form(ctx, case, "helmholtz"), x), ref)


@pytest.mark.parametrize("cell, p, kind", [("hex", 3, "helmholtz"), ("tet", 2, "elasticity"), ("tet", 4, "laplace")])
def test_space_with_library_built_map(ctx, cell, p, kind):
    """mfa_space_create without a map: the library builds it from the mesh; the operator on that map matches the
    oracle on the same map (read back from the space)."""
    mesh = fi.hex_box_mesh(3, perturb=0.1, seed=8) if cell == "hex" else fi.kuhn_tet_mesh(3, perturb=0.1, seed=8)
    ct = 8 if cell == "hex" else 4
    ncomp = 3 if kind == "elasticity" else 1
    m = mfa.Mesh(ctx, ct, mesh.coords, mesh.cell_vert)
    sp = mfa.Space(m, p, ncomp)
    cn = sp.cell_node()
    f = mfa.Form(sp, KIND_NAMES[kind])
    x = fi.uniform_vector(sp.ndof, seed=9)
    qdeg = p + 1 if cell == "hex" else 2 * p
    ref = oracle.Problem(ct, mesh.coords, mesh.cell_vert, p, cn, sp.nnode, KIND_NAMES[kind], ncomp=ncomp,
                         qdeg=qdeg).apply(x)
    y = f.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    compare(y.cpu().numpy(), ref)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
@pytest.mark.parametrize("scatter", ["atomic", "colour"])
def test_hex_on_the_fly_geometry(ctx, p, kind, scatter):
    """Geometry recomputed at every point from the vertices (no stored factors): same operator."""
    nx = {1: 7, 2: 5, 3: 5, 4: 3, 6: 3, 8: 2}[p]
    case = hex_case(nx, p)
    x = fi.uniform_vector(case["nnode"], seed=31)
    ref = oracle_problem(case, kind, k2=0.6).apply(x)
    form = gpu_form(ctx, case, kind, k2=0.6, scatter=SCATTER[scatter], geometry=mfa.MFA_GEOM_ONTHEFLY)
    cfg = form.config()
    assert cfg.geometry == mfa.MFA_GEOM_ONTHEFLY and cfg.variant == mfa.MFA_VARIANT_POINT
    assert all(c.geometry == mfa.MFA_GEOM_ONTHEFLY for c in form.configs())
    compare(run(ctx, form, x), ref)


def test_on_the_fly_geometry_limits(ctx):
    case = hex_case(3, 2)
    form = gpu_form(ctx, case, "helmholtz", geometry=mfa.MFA_GEOM_ONTHEFLY)
    with pytest.raises(mfa.MfaError) as e:
        form.diagonal()
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    stored = mfa.mfa_launch_config(variant=mfa.MFA_VARIANT_POINT, cells_per_block=0, scatter=mfa.MFA_SCATTER_ATOMIC,
                                   geometry=mfa.MFA_GEOM_STORED)
    with pytest.raises(mfa.MfaError) as e:
        form.set_config(stored)  # no stored factors to switch to
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    for kw in [dict(precision=mfa.MFA_PREC_FP32), dict(qdeg=4), dict(scatter=mfa.MFA_SCATTER_WARP)]:
        with pytest.raises(mfa.MfaError) as e:
            gpu_form(ctx, case, "helmholtz", geometry=mfa.MFA_GEOM_ONTHEFLY, **kw)
        assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    # a stored form lists the on-the-fly configuration too, and it gives the same result
    f2 = gpu_form(ctx, case, "helmholtz")
    otf = [c for c in f2.configs() if c.geometry == mfa.MFA_GEOM_ONTHEFLY]
    assert otf
    x = fi.uniform_vector(case["nnode"], seed=32)
    y_stored = run(ctx, f2, x)
    f2.set_config(otf[0])
    compare(run(ctx, f2, x), y_stored, tol=1e-13)
