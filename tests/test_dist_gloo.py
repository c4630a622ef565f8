"""Partitioned operator action and CG on 2 gloo ranks (CPU), local applies by the oracle.

Checks the halo plan and the exchange logic of paper_1903_08243_gb300.dist:
the distributed action equals the single-domain action on every node, and
distributed CG converges to the dense solution.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(kind):
    from tests.problems import hex_case, tet_case, oracle_problem

    if kind == "hex":
        case = hex_case(4, 2)
        return case, oracle_problem(case, "helmholtz")
    case = tet_case(3, 2, ncomp=3, perturb=0.1, seed=4)
    return case, oracle_problem(case, "elasticity")


def _worker(rank, world, port, kind, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1903_08243_gb300 import dist as mdist
        import fe_inputs as fi

        case, pb = _problem(kind)
        nc = case["ncomp"]
        plan = mdist.build_plan(case["cell_node"], case["nnode"], world, rank)
        local = oracle.Problem(case["cell_type"], case["coords"], case["cell_vert"][plan.cells], case["degree"],
                               plan.local_cell_node, plan.l2g.size, pb._s.kind, ncomp=nc, qdeg=pb._s.qdeg)

        def local_apply(xl):
            return torch.from_numpy(local.apply(xl.numpy().reshape(-1)).reshape(xl.shape))

        x = fi.uniform_vector(case["nnode"] * nc, seed=9).reshape(-1, nc)
        xl = torch.from_numpy(x[plan.l2g].copy())
        xl[~torch.from_numpy(plan.owned)] = 0.0  # ghosts must come from the exchange
        y = mdist.distributed_apply(plan, local_apply, xl)
        yref = pb.apply(x.reshape(-1)).reshape(-1, nc)
        err_apply = float(np.abs(y.numpy() - yref[plan.l2g]).max() / np.abs(yref).max())

        err_cg = 0.0
        if kind == "hex":
            A = pb.dense()
            b = fi.uniform_vector(case["nnode"], seed=10)
            xs = np.linalg.solve(A, b)
            bl = torch.from_numpy(b[plan.l2g].copy()).reshape(-1, 1)
            dl = torch.from_numpy(np.diag(A)[plan.l2g].copy()).reshape(-1, 1)
            xl0 = torch.zeros_like(bl)
            xsol, it, res = mdist.distributed_cg(plan, local_apply, bl, xl0, dl, rtol=1e-12, maxit=500)
            err_cg = float(np.abs(xsol.numpy().ravel() - xs[plan.l2g]).max() / np.abs(xs).max())
        out[rank] = (err_apply, err_cg, int(plan.owned.sum()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["hex", "tet"])
def test_partitioned_apply_and_cg_two_ranks(kind):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, kind, out), nprocs=world, join=True, start_method="spawn")
    assert len(out) == world
    for rank in range(world):
        err_apply, err_cg, nowned = out[rank]
        assert err_apply <= 1e-13, err_apply
        assert err_cg <= 1e-8, err_cg
    from tests.problems import hex_case, tet_case

    nnode = hex_case(4, 2)["nnode"] if kind == "hex" else tet_case(3, 2, ncomp=3, perturb=0.1, seed=4)["nnode"]
    assert sum(out[r][2] for r in range(world)) == nnode  # every node owned exactly once


def test_plan_ownership_three_ranks():
    from paper_1903_08243_gb300 import dist as mdist
    from tests.problems import hex_case

    case = hex_case(5, 1)
    plans = [mdist.build_plan(case["cell_node"], case["nnode"], 3, r) for r in range(3)]
    owned = np.zeros(case["nnode"], dtype=int)
    for p in plans:
        owned[p.l2g[p.owned]] += 1
        for peer, ids in p.send_import.items():
            assert np.array_equal(np.sort(plans[peer].l2g[plans[peer].recv_import[p.rank]]), np.sort(p.l2g[ids]))
    assert np.all(owned == 1)
