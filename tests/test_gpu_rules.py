"""GPU parity of the simplex forms with Table 2's fully symmetric rules (MFA_RULE_SYMMETRIC) against the oracle with
the same rules, including the integrands where the rule changes the result (neo-Hookean; St Venant-Kirchhoff below
its polynomial degree), and the point counts the default rule choice gives (Table 2's Q column)."""
import os

import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, oracle_problem, tet_case, tri_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make_form(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def check(ctx, case, kind, x, u=None, symmetric=True, **kw):
    okw = dict(kw)
    ref = oracle_problem(case, kind, ucoef=u if kind == "hyper_jac" else None,
                         rule="symmetric" if symmetric else "collapsed", **okw).apply(x)
    form = make_form(ctx, case, kind, rule=mfa.MFA_RULE_SYMMETRIC if symmetric else mfa.MFA_RULE_AUTO, **kw)
    if kind == "hyper_jac":
        form.set_coefficient(torch.from_numpy(u).cuda())
    y = form.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    y = y.cpu().numpy()
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert rel <= TOL and np.abs(y - ref).max() <= TOL * np.abs(ref).max(), rel
    return form, y


@pytest.mark.parametrize("p", [2, 3, 4])
@pytest.mark.parametrize("kind, law", [("hyper_res", mfa.MFA_LAW_NEOHOOKE), ("hyper_jac", mfa.MFA_LAW_NEOHOOKE),
                                       ("hyper_res", mfa.MFA_LAW_SVK), ("hyper_jac", mfa.MFA_LAW_SVK)])
def test_tet_hyperelastic_symmetric(ctx, p, kind, law):
    case = tet_case(2, p, ncomp=3, perturb=0.1, seed=7)
    u = fi.sinusoid_displacement(case["nodes"], seed=8).ravel()
    x = u if kind == "hyper_res" else fi.uniform_vector(u.size, seed=9)
    kw = dict(lam=1.1, mu=0.8, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.1, -0.05, 0.2)
    form, y = check(ctx, case, kind, x, u, **kw)
    assert form.info().nq == {2: 14, 3: 24, 4: 125}[p]  # rule degree 4, 6 (= qdeg), 8


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind, law", [("hyper_res", mfa.MFA_LAW_NEOHOOKE), ("hyper_jac", mfa.MFA_LAW_SVK)])
def test_tri_hyperelastic_symmetric(ctx, p, kind, law):
    case = tri_case(4, p, ncomp=2, seed=5)
    u = fi.sinusoid_displacement(case["nodes"], seed=10)[:, :2].ravel()
    x = u if kind == "hyper_res" else fi.uniform_vector(u.size, seed=11)
    kw = dict(lam=1.2, mu=0.9, law=law)
    if kind == "hyper_res":
        kw["b"] = (0.05, 0.1, 0.0)
    form, _ = check(ctx, case, kind, x, u, **kw)
    # neo-Hookean: rule degree qdeg = 4, 4, 6, 8; St Venant-Kirchhoff: its degree 4(p - 1) = 0, 4, then qdeg 6, 8
    expect = {1: 6, 2: 6, 3: 12, 4: 25} if law == mfa.MFA_LAW_NEOHOOKE else {1: 1, 2: 6, 3: 12, 4: 25}
    assert form.info().nq == expect[p]


def test_symmetric_rule_changes_a_nonpolynomial_action(ctx):
    """The neo-Hookean residual with 14 and with 27 points: both match their oracle, and they differ."""
    case = tet_case(2, 2, ncomp=3, perturb=0.1, seed=12)
    u = fi.sinusoid_displacement(case["nodes"], seed=13).ravel()
    kw = dict(law=mfa.MFA_LAW_NEOHOOKE)
    f14, y14 = check(ctx, case, "hyper_res", u, u, symmetric=True, **kw)
    f27, y27 = check(ctx, case, "hyper_res", u, u, symmetric=False, **kw)
    assert (f14.info().nq, f27.info().nq) == (14, 27)
    assert np.linalg.norm(y14 - y27) > 1e-10 * np.linalg.norm(y27)


def table2_rows():
    return [l.split() for l in open(os.path.join(HERE, "golden", "table2_simplex_points.txt")) if l[0] != "#"]


@pytest.mark.parametrize("row", table2_rows(), ids=lambda r: "-".join(r))
def test_default_point_counts_are_table2(ctx, row):
    """Polynomial integrands take Table 2's rule by default (exact, so only rounding changes)."""
    cell, form, p, _, q = row
    p, q = int(p), int(q)
    kind = {"mass": "mass", "laplacian": "laplace"}[form]
    case = tet_case(1, p) if cell == "tet" else tri_case(2, p)
    f = make_form(ctx, case, kind)
    assert f.info().nq == q
    x = fi.uniform_vector(case["nnode"], seed=14)
    ref = oracle_problem(case, kind).apply(x)  # the oracle's collapsed rule, exact too
    y = f.apply(torch.from_numpy(x).cuda())
    ctx.sync()
    assert np.linalg.norm(y.cpu().numpy() - ref) <= TOL * np.linalg.norm(ref)


def test_bad_rule_is_rejected(ctx):
    case = tet_case(1, 1)
    with pytest.raises(mfa.MfaError) as e:
        make_form(ctx, case, "mass", rule=7)
    assert e.value.code == mfa.MFA_ERR_ARG
