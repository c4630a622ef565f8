"""Host-buffer applies through the C ABI: mfa_apply_host and the overlapped mfa_apply_host_many give the device
apply's result (and so the oracle's) for forms of different cells and sizes; bad arguments are rejected."""
import numpy as np
import pytest

import fe_inputs as fi
from tests.problems import KIND_NAMES, hex_case, oracle_problem, quad_case, tet_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def make(ctx, case, kind, **kw):
    m = mfa.Mesh(ctx, case["cell_type"], case["coords"], case["cell_vert"])
    sp = mfa.Space(m, case["degree"], case["ncomp"], case["cell_node"], case["nnode"])
    return mfa.Form(sp, KIND_NAMES[kind], **kw)


def problems():
    h = hex_case(6, 3)
    t = tet_case(4, 2, ncomp=3, perturb=0.1, seed=2)
    q = quad_case(9, 4)
    xs = [fi.uniform_vector(h["nnode"], seed=1), fi.uniform_vector(3 * t["nnode"], seed=2),
          fi.uniform_vector(q["nnode"], seed=3)]
    return [(h, "helmholtz", dict(k2=0.7)), (t, "elasticity", dict(lam=1.3, mu=0.6)), (q, "laplace", {})], xs


def test_apply_host_matches_oracle(ctx):
    specs, xs = problems()
    for (case, kind, kw), x in zip(specs, xs):
        f = make(ctx, case, kind, **kw)
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        mfa.mfa_apply_host(ctx.h, f.h, xh, yh)
        ref = oracle_problem(case, kind, **kw).apply(x)
        assert np.linalg.norm(yh.numpy() - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_many_matches_device_apply(ctx, pinned):
    specs, xs = problems()
    forms = [make(ctx, case, kind, **kw) for case, kind, kw in specs]
    hx = [torch.from_numpy(x) for x in xs]
    if pinned:
        hx = [h.pin_memory() for h in hx]
    hy = [torch.full_like(h, np.nan) for h in hx]
    if pinned:
        hy = [h.pin_memory() for h in hy]
    for rep in range(2):  # the second call reuses the staging buffers, streams and events
        mfa.mfa_apply_host_many(ctx.h, [f.h for f in forms], hx, hy)
        for f, x, y in zip(forms, xs, hy):
            yd = f.apply(torch.from_numpy(x).cuda())
            ctx.sync()
            ref = yd.cpu().numpy()
            assert np.linalg.norm(y.numpy() - ref) <= 1e-13 * np.linalg.norm(ref)


def test_apply_host_many_arguments(ctx):
    specs, xs = problems()
    f = make(ctx, *specs[0][:2], **specs[0][2])
    x = torch.from_numpy(xs[0])
    y = torch.empty_like(x)
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_apply_host_many(ctx.h, [f.h, f.h], [x, x], [y, y])
    assert e.value.code == mfa.MFA_ERR_ARG
    mfa.mfa_apply_host_many(ctx.h, [], [], [])  # nothing to do
