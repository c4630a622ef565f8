"""Launch configurations and the autotuner: every compiled configuration of a
form computes the same operator (parity with the FP64 oracle), the tuner times
all of them and keeps the fastest, and invalid choices are refused."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, hex_case, oracle_problem, tet_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

TOL = {mfa.MFA_PREC_FP64: 1e-12, mfa.MFA_PREC_FP32: 1e-5, mfa.MFA_PREC_BF16: 1e-2}


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def rel_err(y, ref):
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


def key(c):
    return (c.variant, c.cells_per_block, c.scatter)


# several batches for every cells-per-block choice, and a ragged last batch
HEX_NX = {1: 9, 3: 5, 4: 5, 5: 4, 6: 4, 8: 3}


@pytest.mark.parametrize("p", [1, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("kind", ["mass", "helmholtz"])
def test_every_fp64_hex_config_matches_oracle(ctx, p, kind):
    case = hex_case(HEX_NX[p], p)
    x = fi.uniform_vector(case["nnode"], seed=41)
    ref = oracle_problem(case, kind, k2=0.5).apply(x)
    form = make_form(ctx, case, kind, k2=0.5)
    cfgs = form.configs()
    variants = {c.variant for c in cfgs}
    assert mfa.MFA_VARIANT_POINT in variants
    assert (mfa.MFA_VARIANT_EVEN_ODD in variants) == (p >= 4)
    assert key(cfgs[0]) == key(form.config())  # the creation-time configuration comes first
    xd = torch.from_numpy(x).cuda()
    for c in cfgs:
        form.set_config(c)
        assert key(form.config()) == key(c)
        y = form.apply(xd)
        ctx.sync()
        assert rel_err(y.cpu().numpy(), ref) <= 1e-12, c.as_dict()


@pytest.mark.parametrize("p", [1, 4, 8])
@pytest.mark.parametrize("prec", [mfa.MFA_PREC_FP32, mfa.MFA_PREC_BF16])
def test_every_mixed_hex_config_matches_oracle(ctx, p, prec):
    case = hex_case(HEX_NX[p], p)
    x = fi.uniform_vector(case["nnode"], seed=42)
    ref = oracle_problem(case, "helmholtz", k2=1.0).apply(x)
    form = make_form(ctx, case, "helmholtz", k2=1.0, precision=prec)
    cfgs = form.configs()
    assert {c.variant for c in cfgs} == {mfa.MFA_VARIANT_LINE, mfa.MFA_VARIANT_LINE_STAGED}
    assert all(c.scatter == mfa.MFA_SCATTER_ATOMIC for c in cfgs)
    xd = torch.from_numpy(x).cuda()
    ys = []
    for c in cfgs:
        form.set_config(c)
        y = form.apply(xd)
        ctx.sync()
        y = y.cpu().numpy()
        assert rel_err(y, ref) <= TOL[prec], c.as_dict()
        ys.append(y)
    # staging moves the same factors: same arithmetic, results equal up to the atomic order
    for y in ys[1:]:
        assert rel_err(y, ys[0]) <= 1e-6


@pytest.mark.parametrize("kind, law", [("elasticity", 0), ("hyper_res", 1), ("hyper_jac", 0)])
def test_every_tet_config_matches_oracle(ctx, kind, law):
    case = tet_case(4, 2, ncomp=3, perturb=0.15, seed=4)
    u = fi.sinusoid_displacement(case["nodes"], seed=2).ravel()  # smooth: J > 0 everywhere
    x = fi.uniform_vector(case["nnode"] * 3, seed=44) if kind == "hyper_jac" else u
    kw = dict(lam=1.0, mu=1.0, law=law)
    prob = oracle_problem(case, kind, ucoef=u if kind == "hyper_jac" else None, **kw)
    ref = prob.apply(x)
    form = make_form(ctx, case, kind, **kw)
    ud = torch.from_numpy(u).cuda()
    if kind == "hyper_jac":
        form.set_coefficient(ud)
    cfgs = form.configs()
    assert sorted({c.cells_per_block for c in cfgs}) == [32, 64, 128]
    xd = torch.from_numpy(x).cuda()
    for c in cfgs:
        form.set_config(c)
        y = form.apply(xd)
        ctx.sync()
        assert rel_err(y.cpu().numpy(), ref) <= 1e-12, c.as_dict()


def test_autotune_times_all_and_keeps_fastest(ctx):
    case = hex_case(8, 4)
    x = fi.uniform_vector(case["nnode"], seed=45)
    ref = oracle_problem(case, "laplace").apply(x)
    form = make_form(ctx, case, "laplace")
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    n_cfg = len(form.configs())
    tried = form.autotune(xd, yd, reps=3)
    assert len(tried) == n_cfg
    times = [c.ms for c in tried]
    assert all(t > 0 for t in times), [c.as_dict() for c in tried]
    best = tried[int(np.argmin(times))]
    chosen = form.config()
    assert key(chosen) == key(best) and chosen.ms == best.ms
    y = form.apply(xd)
    ctx.sync()
    assert rel_err(y.cpu().numpy(), ref) <= 1e-12
    # the work model follows the chosen variant and stays positive
    assert form.info().flops > 0


def test_set_config_refuses_uncompiled_choices(ctx):
    case = hex_case(3, 3)
    form = make_form(ctx, case, "helmholtz")
    bad = mfa.mfa_launch_config(variant=mfa.MFA_VARIANT_POINT, cells_per_block=3, scatter=mfa.MFA_SCATTER_ATOMIC)
    with pytest.raises(mfa.MfaError) as e:
        form.set_config(bad)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED
    mixed_only = mfa.mfa_launch_config(variant=mfa.MFA_VARIANT_LINE, cells_per_block=0, scatter=mfa.MFA_SCATTER_ATOMIC)
    with pytest.raises(mfa.MfaError):
        form.set_config(mixed_only)
    # Q2: no even-odd kernel below n = 5
    form2 = make_form(ctx, hex_case(3, 2), "helmholtz")
    eo = mfa.mfa_launch_config(variant=mfa.MFA_VARIANT_EVEN_ODD, cells_per_block=0, scatter=mfa.MFA_SCATTER_ATOMIC)
    with pytest.raises(mfa.MfaError):
        form2.set_config(eo)
    # AUTO selects the default again
    form.set_config(mfa.mfa_launch_config(variant=mfa.MFA_VARIANT_AUTO, cells_per_block=0,
                                          scatter=mfa.MFA_SCATTER_ATOMIC))
    assert form.config().variant == mfa.MFA_VARIANT_POINT


def test_cells_per_block_at_creation(ctx):
    case = hex_case(5, 3)
    x = fi.uniform_vector(case["nnode"], seed=46)
    ref = oracle_problem(case, "laplace").apply(x)
    form = make_form(ctx, case, "laplace", cells_per_block=8)  # Q3: n^3 = 64 points, default 4
    assert form.config().cells_per_block == 8
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    assert rel_err(y.cpu().numpy(), ref) <= 1e-12
    with pytest.raises(mfa.MfaError) as e:
        make_form(ctx, case, "laplace", cells_per_block=5)
    assert e.value.code == mfa.MFA_ERR_UNSUPPORTED


def test_colour_configs_are_bitwise_deterministic(ctx):
    case = hex_case(6, 4)
    x = torch.from_numpy(fi.uniform_vector(case["nnode"], seed=47)).cuda()
    form = make_form(ctx, case, "helmholtz")
    for c in form.configs():
        if c.scatter != mfa.MFA_SCATTER_COLOUR:
            continue
        form.set_config(c)
        y1 = form.apply(x).clone()
        y2 = form.apply(x)
        ctx.sync()
        assert torch.equal(y1, y2), c.as_dict()
