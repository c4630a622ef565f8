"""GPU parity of the persistent kernels' multi-batch path.

Every apply kernel is a persistent launch: a block takes batch blockIdx.x,
then walks on with a stride of gridDim.x, and several kernels request the next
batch's node indices (or stage its factors) while the current batch runs.  At
the benchmark sizes each block walks tens of batches; the small meshes of the
other parity tests give every block a single one.  Here the grid is capped
(mfa_launch_config.max_blocks = 1 and 3) so that one block walks every batch
of the mesh, and three blocks walk ragged shares, for every compiled
configuration of every kernel family, against the FP64 oracle (Section 2.2's
global assembly).  The 64^3 cases at the end run the dominant kernels of the
benchmark at full size in their default grid, on sampled dofs.

Tolerances: relative L2 error 1e-12 for FP64, 1e-5 for FP32 and 1e-2 for BF16
arithmetic (the stated accuracy targets), and for FP64 also the max-abs error
relative to max|y_ref|.  The BF16 paths round x, the factors and the 1D tables
to 8 significant bits, so a single entry can exceed 1e-2 of max|y_ref| while the
L2 error stays below it.
"""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, cells_touching, hex_case, oracle_problem, quad_case, tet_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

TOL = {mfa.MFA_PREC_FP64: 1e-12, mfa.MFA_PREC_FP32: 1e-5, mfa.MFA_PREC_BF16: 1e-2}
CAPS = (1, 3)


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def compare(y, ref, tol, what=None):
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    mx = np.abs(y - ref).max() / np.abs(ref).max()
    assert rel <= tol, (rel, mx, what)
    if tol <= 1e-12:
        assert mx <= tol, (rel, mx, what)


def every_config_capped(ctx, form, x, ref, tol):
    """Apply with every compiled configuration and each grid cap; returns how many launches were checked."""
    xd = torch.from_numpy(x).cuda()
    checked = 0
    for c in form.configs():
        for cap in CAPS:
            c.max_blocks = cap
            form.set_config(c)
            got = form.config()
            assert (got.variant, got.cells_per_block, got.max_blocks) == (c.variant, c.cells_per_block, cap)
            y = torch.full_like(xd, 3.0)
            form.apply(xd, y)
            ctx.sync()
            compare(y.cpu().numpy(), ref, tol, c.as_dict())
            checked += 1
    return checked


def test_grid_cap_is_validated_and_kept(ctx):
    case = hex_case(3, 2)
    form = make_form(ctx, case, "mass")
    assert form.config().max_blocks == 0
    form.set_max_blocks(2)
    assert form.config().max_blocks == 2
    bad = form.config()
    bad.max_blocks = -1
    with pytest.raises(mfa.MfaError) as e:
        form.set_config(bad)
    assert e.value.code == mfa.MFA_ERR_ARG
    assert form.config().max_blocks == 2
    # the listed configurations carry no cap, and the tuner leaves none
    assert all(c.max_blocks == 0 for c in form.configs())
    xd = torch.from_numpy(fi.uniform_vector(case["nnode"], seed=5)).cuda()
    form.autotune(xd, torch.empty_like(xd), reps=1)
    assert form.config().max_blocks == 0


# ------------------------------------------------------------------ FP64 hexahedra: point, even-odd, colour,
# warp-aggregated and on-the-fly configurations.  nx gives >= 7 batches at the largest cells-per-block choice.
HEX_NX = {1: 7, 2: 5, 3: 4, 4: 4, 5: 4, 6: 4, 7: 3, 8: 3}


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("kind", ["mass", "laplace", "helmholtz"])
def test_fp64_hex_every_config(ctx, p, kind):
    case = hex_case(HEX_NX[p], p, seed=p)
    x = fi.uniform_vector(case["nnode"], seed=60 + p)
    ref = oracle_problem(case, kind, k2=0.7).apply(x)
    form = make_form(ctx, case, kind, k2=0.7)
    variants = {c.variant for c in form.configs()}
    assert (mfa.MFA_VARIANT_EVEN_ODD in variants) == (p >= 4)
    assert every_config_capped(ctx, form, x, ref, 1e-12) >= 2 * len(CAPS)


# ------------------------------------------------------------------ FP32 / BF16 hexahedra: lines with factors from
# global memory and staged by bulk copies (the mbarrier phase alternates from one batch to the next).
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("prec", [mfa.MFA_PREC_FP32, mfa.MFA_PREC_BF16])
@pytest.mark.parametrize("kind", ["mass", "helmholtz"])
def test_mixed_hex_every_config(ctx, p, prec, kind):
    case = hex_case(HEX_NX[p], p, seed=10 + p)
    x = fi.uniform_vector(case["nnode"], seed=70 + p)
    ref = oracle_problem(case, kind, k2=1.0).apply(x)
    form = make_form(ctx, case, kind, k2=1.0, precision=prec)
    assert {c.variant for c in form.configs()} == {mfa.MFA_VARIANT_LINE, mfa.MFA_VARIANT_LINE_STAGED}
    every_config_capped(ctx, form, x, ref, TOL[prec])


@pytest.mark.parametrize("p", [2, 4, 7])
@pytest.mark.parametrize("prec", [mfa.MFA_PREC_FP32, mfa.MFA_PREC_BF16])
def test_mixed_hex_float_vectors_capped(ctx, p, prec):
    """mfa_apply_f32 (float x and y) walks the same batches under the cap."""
    case = hex_case(HEX_NX[p], p, seed=20 + p)
    x = fi.uniform_vector(case["nnode"], seed=80 + p)
    ref = oracle_problem(case, "helmholtz", k2=1.0).apply(x)
    form = make_form(ctx, case, "helmholtz", k2=1.0, precision=prec)
    xf = torch.from_numpy(x).cuda().float()
    for cap in CAPS:
        form.set_max_blocks(cap)
        y = torch.full_like(xf, 2.0)
        mfa.mfa_apply_f32(ctx.h, form.h, xf, y)
        ctx.sync()
        # float vectors add the rounding of x and y to float: 1e-5 covers it (|x| <= 1, ~1e-7 per entry)
        compare(y.double().cpu().numpy(), ref, TOL[prec])


# ------------------------------------------------------------------ grouped persistent launches
def _group_forms(ctx, cap):
    """Three members per class (FP64 point, FP64 even-odd, FP32 and BF16 lines) with different mesh sizes, so a
    block's walk crosses from one member's batches into the next one's."""
    specs = [(2, mfa.MFA_PREC_FP64), (6, mfa.MFA_PREC_FP64), (3, mfa.MFA_PREC_FP32), (4, mfa.MFA_PREC_BF16)]
    forms, xs, refs = [], [], []
    for i, (p, prec) in enumerate(specs):
        for j, nx in enumerate((2, 3, 4) if p <= 4 else (2, 3, 3)):
            case = hex_case(nx, p, seed=300 + 10 * i + j)
            f = make_form(ctx, case, "helmholtz", k2=1.0, precision=prec)
            f.set_max_blocks(cap)
            x = fi.uniform_vector(case["nnode"], seed=400 + 10 * i + j)
            forms.append(f)
            xs.append(torch.from_numpy(x).cuda())
            refs.append((oracle_problem(case, "helmholtz", k2=1.0).apply(x), TOL[prec]))
    return forms, xs, refs


@pytest.mark.parametrize("cap", CAPS)
def test_grouped_launches_capped(ctx, cap):
    forms, xs, refs = _group_forms(ctx, cap)
    ys = [torch.full_like(x, 5.0) for x in xs]
    mfa.mfa_apply_batched(ctx.h, [f.h for f in forms], xs, ys)
    for y, (ref, tol) in zip(ys, refs):
        compare(y.cpu().numpy(), ref, tol)
    # the same batch recorded in a CUDA graph and replayed twice
    ys = [torch.empty_like(x) for x in xs]
    b = mfa.mfa_batch_create(ctx.h, [f.h for f in forms], xs, ys)
    try:
        assert mfa.mfa_batch_info(b) == (4, 0)
        for y in ys:
            y.fill_(-1.0)
        for _ in range(2):
            mfa.mfa_batch_apply(ctx.h, b)
        ctx.sync()
        for y, (ref, tol) in zip(ys, refs):
            compare(y.cpu().numpy(), ref, tol)
    finally:
        mfa.mfa_batch_destroy(b)


# ------------------------------------------------------------------ vector hexahedra, quadrilaterals, simplices
def _vector_inputs(case, kind, seed, ncomp):
    u = fi.sinusoid_displacement(case["nodes"], seed=seed)[:, :ncomp].ravel()  # smooth: J > 0
    x = u if kind == "hyper_res" else fi.uniform_vector(u.size, seed=seed + 50)
    return u, x


def _check_vector(ctx, case, kind, law, seed, **extra):
    nc = case["ncomp"]
    kw = dict(lam=1.1, mu=0.8, law=law)
    if nc > 1:
        u, x = _vector_inputs(case, kind, seed, nc)
    else:
        u, x = None, fi.uniform_vector(case["nnode"], seed=seed)
        kw = dict(k2=0.9)
    ref = oracle_problem(case, kind, ucoef=u if kind == "hyper_jac" else None, **kw).apply(x)
    form = make_form(ctx, case, kind, **kw, **extra)
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    return every_config_capped(ctx, form, x, ref, 1e-12)


@pytest.mark.parametrize("p, kind, law", [(1, "elasticity", 0), (2, "hyper_res", mfa.MFA_LAW_NEOHOOKE),
                                          (2, "hyper_jac", mfa.MFA_LAW_SVK), (3, "laplace", 0)])
def test_hex_vector_capped(ctx, p, kind, law):
    _check_vector(ctx, hex_case({1: 5, 2: 3, 3: 3}[p], p, ncomp=3, seed=30 + p), kind, law, seed=p)


@pytest.mark.parametrize("p, kind, ncomp", [(1, "helmholtz", 1), (3, "helmholtz", 1), (2, "elasticity", 2),
                                            (2, "hyper_res", 2)])
def test_quad_capped(ctx, p, kind, ncomp):
    _check_vector(ctx, quad_case({1: 24, 2: 10, 3: 8}[p], p, ncomp=ncomp), kind, mfa.MFA_LAW_NEOHOOKE, seed=40 + p)


@pytest.mark.parametrize("p, kind, ncomp", [(1, "mass", 1), (2, "helmholtz", 1), (2, "elasticity", 3),
                                            (2, "hyper_res", 3), (3, "helmholtz", 1), (4, "elasticity", 3)])
def test_tet_capped(ctx, p, kind, ncomp):
    # P1/P2: one thread per cell (32/64/128-thread blocks); P3+: one warp per cell
    _check_vector(ctx, tet_case({1: 6, 2: 4, 3: 3, 4: 2}[p], p, ncomp=ncomp, perturb=0.1, seed=50 + p), kind,
                  mfa.MFA_LAW_NEOHOOKE, seed=50 + p)


@pytest.mark.parametrize("p, kind, ncomp", [(1, "mass", 1), (3, "helmholtz", 1), (2, "elasticity", 2),
                                            (5, "helmholtz", 1)])
def test_tri_capped(ctx, p, kind, ncomp):
    # P1..P4: one thread per cell; P5: one warp per cell
    _check_vector(ctx, tri_case({1: 16, 2: 8, 3: 8, 5: 4}[p], p, ncomp=ncomp), kind, mfa.MFA_LAW_SVK, seed=60 + p)


# ------------------------------------------------------------------ full size: the benchmark's dominant kernels
def _sampled(case, y, x, kind, prec, seed, ndof=64):
    rng = np.random.default_rng(seed)
    dofs = rng.choice(case["nnode"], size=ndof, replace=False)
    cells = cells_touching(case["cell_node"], dofs)
    ref = oracle_problem(case, kind, k2=1.0).apply(x, cells=cells)
    compare(y[dofs], ref[dofs], TOL[prec])


def test_full_size_q6_helmholtz_even_odd(ctx):
    """64^3 Q6 Helmholtz (57 M dofs) by the even-odd kernel in the benchmark's launch configuration: ~86 batches
    per block, every one through the next-batch node prefetch."""
    case = hex_case(64, 6)
    x = fi.uniform_vector(case["nnode"], seed=1)
    form = make_form(ctx, case, "helmholtz", k2=1.0)
    assert form.config().variant == mfa.MFA_VARIANT_EVEN_ODD and form.config().max_blocks == 0
    xd = torch.from_numpy(x).cuda()
    y = form.apply(xd)
    ctx.sync()
    _sampled(case, y.cpu().numpy(), x, "helmholtz", mfa.MFA_PREC_FP64, seed=6)
    del xd, y


@pytest.mark.parametrize("prec", [mfa.MFA_PREC_FP32, mfa.MFA_PREC_BF16])
def test_full_size_q4_helmholtz_staged_lines(ctx, prec):
    """64^3 Q4 Helmholtz (17 M dofs) by the staged line kernel: the factor staging alternates its mbarrier phase
    over ~100 batches per block."""
    case = hex_case(64, 4)
    x = fi.uniform_vector(case["nnode"], seed=1)
    form = make_form(ctx, case, "helmholtz", k2=1.0, precision=prec)
    staged = [c for c in form.configs() if c.variant == mfa.MFA_VARIANT_LINE_STAGED]
    assert staged
    xd = torch.from_numpy(x).cuda()
    for c in staged:
        form.set_config(c)
        y = form.apply(xd)
        ctx.sync()
        _sampled(case, y.cpu().numpy(), x, "helmholtz", prec, seed=4)
