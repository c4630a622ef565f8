"""Pins of the preconditioner oracle: Jacobi reduction, homogeneity, and finite-difference gradients."""
import numpy as np
import pytest

import fe_inputs as fi
from oracle import precond as op
from tests.problems import hex_case, oracle_problem


@pytest.fixture(scope="module")
def small():
    case = hex_case(3, 2)
    pb = oracle_problem(case, "helmholtz")
    A = pb.dense()
    n = case["nnode"]
    nloc = case["cell_node"].shape[1]
    rng = np.random.default_rng(0)
    W1 = rng.uniform(-0.3, 0.3, (16, nloc))
    b1 = rng.uniform(-0.1, 0.1, 16)
    W2 = rng.uniform(-0.3, 0.3, (nloc, 16)) * 1e-2
    winv = op.multiplicity_weights(case["cell_node"], n)
    dinv = 1.0 / np.diag(A)
    e = fi.uniform_vector(n, seed=5)
    r = A @ e
    return case, A, W1, b1, W2, winv, dinv, r, e


def test_zero_network_is_jacobi(small):
    case, A, W1, b1, W2, winv, dinv, r, e = small
    z = op.apply(r, case["cell_node"], winv, dinv, W1, b1, 0 * W2)
    np.testing.assert_allclose(z, dinv * r, rtol=0, atol=0)


def test_positive_homogeneity(small):
    case, A, W1, b1, W2, winv, dinv, r, e = small
    z1 = op.apply(r, case["cell_node"], winv, dinv, W1, b1, W2)
    z3 = op.apply(3.0 * r, case["cell_node"], winv, dinv, W1, b1, W2)
    np.testing.assert_allclose(z3, 3.0 * z1, rtol=1e-13, atol=1e-15)


def test_partition_of_unity_weights(small):
    case = small[0]
    winv = op.multiplicity_weights(case["cell_node"], case["nnode"])
    acc = np.zeros(case["nnode"])
    np.add.at(acc, case["cell_node"], winv[case["cell_node"]])
    np.testing.assert_allclose(acc, 1.0, rtol=1e-15)


def test_gradients_match_finite_differences(small):
    case, A, W1, b1, W2, winv, dinv, r, e = small
    cn = case["cell_node"]
    L, dW1, db1, dW2 = op.loss_and_grad(r, e, lambda v: A @ v, cn, winv, dinv, W1, b1, W2)
    rng = np.random.default_rng(1)
    for name, P, G in [("W1", W1, dW1), ("b1", b1, db1), ("W2", W2, dW2)]:
        D = rng.standard_normal(P.shape)
        eps = 1e-6

        def loss_at(Q):
            args = {"W1": W1, "b1": b1, "W2": W2}
            args[name] = Q
            return op.loss_and_grad(r, e, lambda v: A @ v, cn, winv, dinv, args["W1"], args["b1"], args["W2"])[0]

        fd = (loss_at(P + eps * D) - loss_at(P - eps * D)) / (2 * eps)
        assert abs(fd - np.sum(G * D)) <= 1e-6 * max(1.0, abs(fd)), (name, fd, np.sum(G * D))
    # the loss is the relative A-norm error of the preconditioned step
    z = op.apply(r, cn, winv, dinv, W1, b1, W2)
    assert abs(L - (z - e) @ A @ (z - e) / (e @ A @ e)) < 1e-13


def test_linear_variant_is_symmetric_positive_definite_and_linear(small):
    case, A, W1, b1, W2, winv, dinv, r, e = small
    cn = case["cell_node"]
    n = case["nnode"]
    Mmat = np.stack([op.apply_linear(np.eye(n)[j], cn, winv, dinv, W1) for j in range(n)], axis=1)
    np.testing.assert_allclose(Mmat, Mmat.T, rtol=0, atol=1e-14 * np.abs(Mmat).max())
    assert np.linalg.eigvalsh(Mmat).min() > 0
    np.testing.assert_allclose(op.apply_linear(r, cn, winv, dinv, W1), Mmat @ r, rtol=1e-12)
    np.testing.assert_allclose(op.apply_linear(r, cn, winv, dinv, 0 * W1), dinv * r, rtol=0, atol=0)


def test_linear_variant_gradient_matches_finite_differences(small):
    case, A, W1, b1, W2, winv, dinv, r, e = small
    cn = case["cell_node"]
    L, dW1 = op.loss_and_grad_linear(r, e, lambda v: A @ v, cn, winv, dinv, W1)
    D = np.random.default_rng(2).standard_normal(W1.shape)
    eps = 1e-6
    fd = (op.loss_and_grad_linear(r, e, lambda v: A @ v, cn, winv, dinv, W1 + eps * D)[0] -
          op.loss_and_grad_linear(r, e, lambda v: A @ v, cn, winv, dinv, W1 - eps * D)[0]) / (2 * eps)
    assert abs(fd - np.sum(dW1 * D)) <= 1e-6 * max(1.0, abs(fd))


def _golden(name):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "precond_hand_worked.txt")
    for line in open(path):
        if line.startswith(name + ":"):
            return np.array([float(v) for v in line.split(":")[1].split()])
    raise KeyError(name)


def test_hand_worked_forward():
    """A case evaluated by hand (tests/golden/precond_hand_worked.txt): the bias, the activation cutting one unit,
    the scaling by s_K, the partition-of-unity weights and the zero-residual cell each change the result, so a
    dropped or misplaced term fails here."""
    cn = np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int32)
    winv = op.multiplicity_weights(cn, 4)
    np.testing.assert_array_equal(winv, [1.0, 0.5, 0.5, 1.0])
    dinv = np.array([0.5, 0.25, 1.0, 2.0])
    r = np.array([3.0, 4.0, 0.0, 0.0])
    W1 = np.array([[1.0, 2.0], [-2.0, 1.0]])
    b1 = np.array([-0.5, 0.5])
    W2 = np.array([[1.0, -1.0], [2.0, 3.0]])
    np.testing.assert_allclose(op.apply(r, cn, winv, dinv, W1, b1, W2), _golden("mlp"), rtol=0, atol=1e-14)
    W1l = np.array([[1.0, 2.0], [0.0, 1.0]])
    np.testing.assert_allclose(op.apply_linear(r, cn, winv, dinv, W1l), _golden("linear"), rtol=0, atol=1e-14)
