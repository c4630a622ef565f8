"""Reverse Cuthill-McKee renumbering (host code of the library, no GPU): valid permutations, restored locality on
a shuffled mesh, and an operator that is unchanged up to the permutation (checked with the oracle)."""
import numpy as np
import pytest

import fe_inputs as fi
import oracle
import paper_1903_08243_gb300 as mfa
from tests.problems import oracle_problem, tet_case


def spread(cell_node):
    """Largest spread of node ids within one cell (a bandwidth proxy)."""
    return int((cell_node.max(axis=1) - cell_node.min(axis=1)).max())


def window(cell_node, block=32):
    """Mean number of distinct 64-node windows touched by a block of consecutive cells."""
    nb = cell_node.shape[0] // block
    w = cell_node[: nb * block].reshape(nb, -1) // 64
    return float(np.mean([np.unique(r).size for r in w]))


@pytest.mark.parametrize("p", [1, 2])
def test_rcm_restores_locality_of_a_shuffled_hex_mesh(p):
    nx = 8
    mesh = fi.hex_box_mesh(nx)
    cn, nnode = fi.hex_node_map(nx, p)
    cv_s, cn_s, _ = fi.shuffle_mesh(mesh.cell_vert, cn, nnode, seed=5)
    # vertices are numbered like the Q1 nodes; shuffle them consistently with a Q1 map
    order, perm = mfa.mfa_order_rcm(cv_s, cn_s, nnode, nvert=mesh.nvert)
    assert np.array_equal(np.sort(order), np.arange(order.size))
    assert np.array_equal(np.sort(perm), np.arange(nnode))
    cv_r, cn_r = mfa.apply_order(cv_s, cn_s, order, perm)
    # a block of 32 consecutive cells touches about as few 64-node windows as with the lexicographic numbering
    # (RCM levels are shells around a corner, so the bandwidth itself is a few times the lexicographic one)
    assert window(cn_r) <= 1.6 * window(cn)
    assert window(cn_r) < window(cn_s) / 3
    assert spread(cn_r) < spread(cn_s) / 1.5


def test_rcm_operator_is_the_permuted_operator():
    case = tet_case(3, 2, ncomp=3, perturb=0.15, seed=3, shuffle=True)
    order, perm = mfa.mfa_order_rcm(case["cell_vert"], case["cell_node"], case["nnode"], nvert=len(case["coords"]))
    cv_r, cn_r = mfa.apply_order(case["cell_vert"], case["cell_node"], order, perm)
    x = fi.uniform_vector(case["nnode"] * 3, seed=4).reshape(-1, 3)
    y = oracle_problem(case, "elasticity").apply(x.ravel()).reshape(-1, 3)
    case_r = dict(case, cell_vert=cv_r, cell_node=cn_r)
    x_r = np.empty_like(x)
    x_r[perm] = x
    y_r = oracle_problem(case_r, "elasticity").apply(x_r.ravel()).reshape(-1, 3)
    np.testing.assert_allclose(y_r[perm], y, rtol=1e-12, atol=1e-14 * np.abs(y).max())


def test_rcm_handles_components_empty_meshes_and_bad_indices():
    # two disjoint tets and an unused node
    cv = np.array([[0, 1, 2, 3], [4, 5, 6, 7]], dtype=np.int32)
    order, perm = mfa.mfa_order_rcm(cv, cv, 9, nvert=8)
    assert sorted(order) == [0, 1] and sorted(perm) == list(range(9))
    assert perm[8] == 8  # a node of no cell keeps a place at the end
    e_order, e_perm = mfa.mfa_order_rcm(np.zeros((0, 4), np.int32), np.zeros((0, 4), np.int32), 0, nvert=0)
    assert e_order.size == 0 and e_perm.size == 0
    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_order_rcm(cv, cv + 5, 9, nvert=8)  # node 12 outside [0, 9)
    assert e.value.code == mfa.MFA_ERR_RANGE
