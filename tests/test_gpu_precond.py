"""Learned preconditioner on the GPU against the FP64 oracle (oracle/precond.py)."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import precond as op
from tests.problems import hex_case, oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


def bf16_round(a):
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


def to_f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# The kernels multiply BF16 operands (weights, Z and H forward, dL/dO and dL/dH backward) with FP32 accumulation;
# the oracle is evaluated with the same operands rounded to BF16 (its `rnd` argument) and the FP32 inputs r, e.
# What remains is FP32 accumulation over <= 128 products (<= 128 * 2^-24 ~ 8e-6 relative) and the few operands
# whose FP32 and FP64 values fall on different sides of a BF16 rounding boundary (one BF16 unit in the last
# place, 2^-8 ~ 4e-3 relative, on roughly one operand in 10^3): together well below 1e-3 of the result.
OPERAND_TOL = 1e-3


def setup(ctx, nx, p, seed=0, w2scale=0.05):
    case = hex_case(nx, p)
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, p, 1, case["cell_node"], case["nnode"])
    f64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    f32 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, precision=mfa.MFA_PREC_FP32)
    pc = mfa.mfa_precond_create(ctx.h, f64.h, seed)
    nloc = (p + 1) ** 3
    rng = np.random.default_rng(seed + 1)
    W1, b1, _ = mfa.unpack_precond_weights(mfa.mfa_precond_get_weights(pc), nloc)
    b1 = rng.uniform(-0.1, 0.1, 128).astype(np.float32)
    W2 = (w2scale * rng.standard_normal((nloc, 128))).astype(np.float32)
    mfa.mfa_precond_set_weights(pc, mfa.pack_precond_weights(W1, b1, W2))
    keep = (m, sp, f64, f32)
    return case, keep, pc, W1.astype(np.float64), b1.astype(np.float64), W2.astype(np.float64)


@pytest.mark.parametrize("nx,p", [(5, 1), (4, 2), (3, 3), (3, 4)])
def test_precond_forward_matches_oracle(ctx, nx, p):
    case, keep, pc, W1, b1, W2 = setup(ctx, nx, p)
    pb = oracle_problem(case, "helmholtz")
    A = pb.dense() if case["nnode"] <= 4000 else None
    dinv = 1.0 / (np.diag(A) if A is not None else None)
    winv = op.multiplicity_weights(case["cell_node"], case["nnode"])
    r = to_f32(fi.uniform_vector(case["nnode"], seed=3))
    dinv = to_f32(dinv)
    # the kernels run the MLP on bfloat16 weights and operands
    ref = op.apply(r, case["cell_node"], winv, dinv, bf16_round(W1), b1, bf16_round(W2), rnd=bf16_round)
    rd = torch.from_numpy(r).float().cuda()
    z = torch.empty_like(rd)
    mfa.mfa_precond_apply(ctx.h, pc, rd, z)
    ctx.sync()
    zg = z.double().cpu().numpy()
    net_ref, net = ref - dinv * r, zg - dinv * r
    err = np.linalg.norm(net - net_ref) / np.linalg.norm(net_ref)
    assert err <= OPERAND_TOL, err
    assert np.linalg.norm(zg - ref) <= OPERAND_TOL * np.linalg.norm(ref)
    mfa.mfa_precond_destroy(pc)


def test_untrained_precond_is_jacobi(ctx):
    case = hex_case(3, 4)
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, 4, 1, case["cell_node"], case["nnode"])
    f64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    pc = mfa.mfa_precond_create(ctx.h, f64.h, 7)
    d = f64.diagonal()
    r = torch.from_numpy(fi.uniform_vector(case["nnode"], seed=4)).float().cuda()
    z = torch.empty_like(r)
    mfa.mfa_precond_apply(ctx.h, pc, r, z)
    ctx.sync()
    ref = (r.double() / d).float()
    assert torch.allclose(z, ref, rtol=1e-6, atol=0)
    mfa.mfa_precond_destroy(pc)


def test_precond_gradient_matches_oracle(ctx):
    nx, p = 3, 2
    case, keep, pc, W1, b1, W2 = setup(ctx, nx, p, w2scale=0.2)
    A = oracle_problem(case, "helmholtz").dense()
    winv = op.multiplicity_weights(case["cell_node"], case["nnode"])
    dinv = 1.0 / np.diag(A)
    e = to_f32(fi.uniform_vector(case["nnode"], seed=6))
    r = to_f32(A @ e)
    L, dW1, db1, dW2 = op.loss_and_grad(r, e, lambda v: A @ v, case["cell_node"], winv, to_f32(dinv), bf16_round(W1),
                                        b1, bf16_round(W2), rnd=bf16_round)
    loss, g = mfa.mfa_precond_loss_grad(ctx.h, pc, keep[3].h, torch.from_numpy(r).float().cuda(),
                                        torch.from_numpy(e).float().cuda())
    gW1, gb1, gW2 = mfa.unpack_precond_weights(g, (p + 1) ** 3)
    # the loss goes through the FP32 operator (relative error ~1e-6) instead of the dense FP64 matrix
    assert abs(loss - L) <= 1e-4 * L, (loss, L)
    for name, ref, got in [("W1", dW1, gW1), ("b1", db1, gb1), ("W2", dW2, gW2)]:
        got = got.astype(np.float64)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2 * OPERAND_TOL, (name, err)
    mfa.mfa_precond_destroy(pc)


def _pairs(ctx, A, f64, nnode, nrhs=2, its=(2, 6, 20)):
    """(r, e) pairs from plain CG iterates: e = x* - x_k, r = b - A x_k."""
    rs, es = [], []
    for j in range(nrhs):
        b = fi.uniform_vector(nnode, seed=50 + j)
        xs = np.linalg.solve(A, b)
        bd = torch.from_numpy(b).cuda()
        for k in its:
            x = torch.zeros_like(bd)
            f64.cg(bd, x, precond=mfa.MFA_PC_NONE, rtol=1e-30, maxit=k)
            xk = x.cpu().numpy()
            rs.append(torch.from_numpy(b - A @ xk).float().cuda())
            es.append(torch.from_numpy(xs - xk).float().cuda())
    return rs, es


def test_training_reduces_the_loss_and_learned_fcg_converges(ctx, tmp_path):
    nx, p = 4, 3
    case = hex_case(nx, p)
    A = oracle_problem(case, "helmholtz").dense()
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, p, 1, case["cell_node"], case["nnode"])
    f64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    f32 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, precision=mfa.MFA_PREC_FP32)
    pc = mfa.mfa_precond_create(ctx.h, f64.h, 11)
    rs, es = _pairs(ctx, A, f64, case["nnode"], nrhs=3, its=(2, 6, 20, 60, 150))
    first, last = mfa.mfa_precond_train(ctx.h, pc, f32.h, rs, es, 600, 5e-4)
    assert last < 0.9 * first, (first, last)  # the network improves on the Jacobi step (first = Jacobi's loss)
    # save / load round trip
    path = tmp_path / "pc.bin"
    mfa.mfa_precond_save(pc, path)
    w = mfa.mfa_precond_get_weights(pc)
    pc2 = mfa.mfa_precond_create(ctx.h, f64.h, 99)
    mfa.mfa_precond_load(pc2, path)
    assert np.array_equal(w, mfa.mfa_precond_get_weights(pc2))
    # the learned flexible CG reaches the FP64 tolerance, on its own and with the Jacobi fallback
    b = fi.uniform_vector(case["nnode"], seed=77)
    bd = torch.from_numpy(b).cuda()
    for fallback in (False, True):
        x = torch.zeros_like(bd)
        rc, it, inn, rel, fb = mfa.mfa_fcg_learned(ctx.h, f64.h, f32.h, pc, 4, bd, x, 1e-10, 1000, fallback=fallback)
        assert rc == mfa.MFA_OK and rel <= 1e-10
        assert fb in ((0,) if not fallback else (0, 1))
        assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 2e-10 * np.linalg.norm(b)
    mfa.mfa_precond_destroy(pc)
    mfa.mfa_precond_destroy(pc2)



# ------------------------------------------------------------------ linear (SPD) variant

def test_linear_precond_forward_and_gradient_match_oracle(ctx):
    nx, p = 3, 3
    case = hex_case(nx, p)
    A = oracle_problem(case, "helmholtz").dense()
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, p, 1, case["cell_node"], case["nnode"])
    f64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    f32 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, precision=mfa.MFA_PREC_FP32)
    pc = mfa.mfa_precond_create(ctx.h, f64.h, 3, mode=mfa.MFA_PRECOND_LINEAR)
    nloc = (p + 1) ** 3
    W1 = (0.3 * np.random.default_rng(4).standard_normal((128, nloc))).astype(np.float32)
    mfa.mfa_precond_set_weights(pc, mfa.pack_precond_weights(W1, np.zeros(128), np.zeros((nloc, 128))))
    winv = op.multiplicity_weights(case["cell_node"], case["nnode"])
    dinv = 1.0 / np.diag(A)
    r = to_f32(fi.uniform_vector(case["nnode"], seed=8))
    W1b = bf16_round(W1)
    ref = op.apply_linear(r, case["cell_node"], to_f32(winv), to_f32(dinv), W1b, rnd=bf16_round)
    z = torch.empty(case["nnode"], dtype=torch.float32, device="cuda")
    mfa.mfa_precond_apply(ctx.h, pc, torch.from_numpy(r).float().cuda(), z)
    ctx.sync()
    zg = z.double().cpu().numpy()
    net = ref - to_f32(dinv) * r
    err = np.linalg.norm((zg - to_f32(dinv) * r) - net) / np.linalg.norm(net)
    assert err <= OPERAND_TOL, err
    e = fi.uniform_vector(case["nnode"], seed=9)
    rr = A @ e
    L, dW1 = op.loss_and_grad_linear(rr, e, lambda v: A @ v, case["cell_node"], winv, dinv, W1b)
    loss, g = mfa.mfa_precond_loss_grad(ctx.h, pc, f32.h, torch.from_numpy(rr).float().cuda(),
                                        torch.from_numpy(e).float().cuda())
    gW1, gb1, gW2 = mfa.unpack_precond_weights(g, nloc)
    assert abs(loss - L) <= 2e-2 * L
    cos = (dW1.ravel() @ gW1.ravel()) / (np.linalg.norm(dW1) * np.linalg.norm(gW1))
    assert cos > 0.999 and np.linalg.norm(gW1 - dW1) <= 5e-2 * np.linalg.norm(dW1)
    assert not gb1.any() and not gW2.any()
    mfa.mfa_precond_destroy(pc)


def test_linear_precond_forward_many_tiles(ctx):
    """The linear mode's forward kernel on 46,656 cells (365 tiles of 128 cells: more tiles than resident blocks,
    so blocks walk several, and a ragged last tile) against the oracle at the kernels' operand precision."""
    case = hex_case(36, 1)
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, 1, 1, case["cell_node"], case["nnode"])
    f64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    pc = mfa.mfa_precond_create(ctx.h, f64.h, 3, mode=mfa.MFA_PRECOND_LINEAR)
    W1 = (0.3 * np.random.default_rng(5).standard_normal((128, 8))).astype(np.float32)
    mfa.mfa_precond_set_weights(pc, mfa.pack_precond_weights(W1, np.zeros(128), np.zeros((8, 128))))
    d = f64.diagonal()
    ctx.sync()
    dinv = to_f32(1.0 / d.cpu().numpy())
    winv = to_f32(op.multiplicity_weights(case["cell_node"], case["nnode"]))
    r = to_f32(fi.uniform_vector(case["nnode"], seed=12))
    ref = op.apply_linear(r, case["cell_node"], winv, dinv, bf16_round(W1), rnd=bf16_round)
    z = torch.empty(case["nnode"], dtype=torch.float32, device="cuda")
    mfa.mfa_precond_apply(ctx.h, pc, torch.from_numpy(r).float().cuda(), z)
    ctx.sync()
    net, got = ref - dinv * r, z.double().cpu().numpy() - dinv * r
    err = np.linalg.norm(got - net) / np.linalg.norm(net)
    assert err <= OPERAND_TOL, err
    mfa.mfa_precond_destroy(pc)


def test_linear_learned_pcg_beats_jacobi_inner_loop(ctx):
    """What training buys: fewer outer iterations than the same solver with the Jacobi inner loop."""
    nx, p = 4, 3
    case = hex_case(nx, p)
    A = oracle_problem(case, "helmholtz").dense()
    m = mfa.Mesh(ctx, 8, case["coords"], case["cell_vert"])
    sp = mfa.Space(m, p, 1, case["cell_node"], case["nnode"])
    f64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ)
    f32 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, precision=mfa.MFA_PREC_FP32)
    pc = mfa.mfa_precond_create(ctx.h, f64.h, 5, mode=mfa.MFA_PRECOND_LINEAR)
    rs, es = _pairs(ctx, A, f64, case["nnode"], nrhs=3, its=(2, 6, 20, 60, 150))
    first, last = mfa.mfa_precond_train(ctx.h, pc, f32.h, rs, es, 800, 2e-3)
    assert last < first
    b = fi.uniform_vector(case["nnode"], seed=78)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    rc, it_l, _, rel, fb = mfa.mfa_fcg_learned(ctx.h, f64.h, f32.h, pc, 4, bd, x, 1e-10, 1000, fallback=False)
    assert rc == mfa.MFA_OK and rel <= 1e-10
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 2e-10 * np.linalg.norm(b)
    rc, it_j, _, _ = mfa.mfa_fcg_mixed(ctx.h, f64.h, f32.h, 4, bd, torch.zeros_like(bd), 1e-10, 1000)
    print("linear learned outer iterations", it_l, "jacobi", it_j, "loss", first, "->", last)
    assert it_l <= it_j
    mfa.mfa_precond_destroy(pc)
