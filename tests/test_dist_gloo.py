"""Partitioned operator action and CG on 2 gloo ranks (CPU), local applies by the oracle.

Checks the halo plan and the exchange logic of paper_1903_08243_gb300.dist:
the distributed action (plain, and boundary cells first with the reverse
exchange overlapping the interior cells) equals the single-domain action on
every node, and distributed CG converges to the dense solution.
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


class HostHaloOps:
    """Stand-in for the library's halo kernels (mfa_halo_pack / mfa_halo_unpack) on the CPU tensors of gloo
    ranks: the same three moves, written with torch indexing (test infrastructure only)."""

    def pack(self, ids, v):
        return v[torch.as_tensor(ids)].contiguous()

    def put(self, ids, buf, v):
        v[torch.as_tensor(ids)] = buf

    def add(self, ids, buf, v):
        v.index_add_(0, torch.as_tensor(ids), buf)


def _problem(kind):
    from tests.problems import hex_case, tet_case, oracle_problem

    if kind == "hex":
        case = hex_case(4, 2)
        return case, oracle_problem(case, "helmholtz")
    if kind == "hex-shuffled-rcb":
        case = hex_case(4, 2, shuffle=True)
        return case, oracle_problem(case, "helmholtz")
    case = tet_case(4, 2, ncomp=3, perturb=0.1, seed=4)  # 4^3: each rank keeps interior cells
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
        parts = mdist.rcb_partition(case["coords"], case["cell_vert"], world) if kind.endswith("rcb") else None
        plan = mdist.build_plan(case["cell_node"], case["nnode"], world, rank, parts)
        local = oracle.Problem(case["cell_type"], case["coords"], case["cell_vert"][plan.cells], case["degree"],
                               plan.local_cell_node, plan.l2g.size, pb._s.kind, ncomp=nc, qdeg=pb._s.qdeg)

        def local_apply(xl):
            return torch.from_numpy(local.apply(xl.numpy().reshape(-1)).reshape(xl.shape))

        x = fi.uniform_vector(case["nnode"] * nc, seed=9).reshape(-1, nc)
        xl = torch.from_numpy(x[plan.l2g].copy())
        xl[~torch.from_numpy(plan.owned)] = 0.0  # ghosts must come from the exchange
        ops = HostHaloOps()
        y = mdist.distributed_apply(plan, local_apply, xl, ops)
        yref = pb.apply(x.reshape(-1)).reshape(-1, nc)
        err_apply = float(np.abs(y.numpy() - yref[plan.l2g]).max() / np.abs(yref).max())

        # boundary cells first, the reverse exchange in flight during the interior cells
        parts = {}
        for name, sel in (("boundary", plan.boundary_cells), ("interior", plan.interior_cells)):
            parts[name] = oracle.Problem(case["cell_type"], case["coords"], case["cell_vert"][plan.cells[sel]],
                                         case["degree"], np.ascontiguousarray(plan.local_cell_node[sel]),
                                         plan.l2g.size, pb._s.kind, ncomp=nc, qdeg=pb._s.qdeg)

        def apply_boundary(xl_, y_=None):
            return torch.from_numpy(parts["boundary"].apply(xl_.numpy().reshape(-1)).reshape(xl_.shape))

        def apply_interior(xl_, y_):
            y_ += torch.from_numpy(parts["interior"].apply(xl_.numpy().reshape(-1)).reshape(xl_.shape))

        xl2 = torch.from_numpy(x[plan.l2g].copy())
        xl2[~torch.from_numpy(plan.owned)] = 0.0
        y2 = mdist.distributed_apply_overlapped(plan, apply_boundary, apply_interior, xl2, ops)
        err_apply = max(err_apply, float(np.abs(y2.numpy() - yref[plan.l2g]).max() / np.abs(yref).max()))
        # interior cells touch no node shared with the other rank, and the two parts cover every cell once
        shared = np.zeros(plan.l2g.size, dtype=bool)
        for ids in list(plan.send_import.values()) + list(plan.recv_import.values()):
            shared[ids] = True
        split_ok = (not shared[plan.local_cell_node[plan.interior_cells]].any() and len(plan.interior_cells) > 0 and
                    np.array_equal(np.sort(np.concatenate([plan.boundary_cells, plan.interior_cells])),
                                   np.arange(len(plan.cells))))

        err_cg = 0.0
        if kind.startswith("hex"):
            A = pb.dense()
            b = fi.uniform_vector(case["nnode"], seed=10)
            xs = np.linalg.solve(A, b)
            bl = torch.from_numpy(b[plan.l2g].copy()).reshape(-1, 1)
            dl = torch.from_numpy(np.diag(A)[plan.l2g].copy()).reshape(-1, 1)
            xl0 = torch.zeros_like(bl)
            xsol, it, res = mdist.distributed_cg(plan, local_apply, bl, xl0, ops, dl, rtol=1e-12, maxit=500)
            err_cg = float(np.abs(xsol.numpy().ravel() - xs[plan.l2g]).max() / np.abs(xs).max())
            xsol2, it2, res2 = mdist.distributed_cg(plan, None, bl, torch.zeros_like(bl), ops, dl, rtol=1e-12,
                                                    maxit=500, overlapped=(apply_boundary, apply_interior))
            err_cg = max(err_cg, float(np.abs(xsol2.numpy().ravel() - xs[plan.l2g]).max() / np.abs(xs).max()))
        out[rank] = (err_apply, err_cg, int(plan.owned.sum()), bool(split_ok))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["hex", "tet", "hex-shuffled-rcb"])
def test_partitioned_apply_and_cg_two_ranks(kind):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, kind, out), nprocs=world, join=True, start_method="spawn")
    assert len(out) == world
    for rank in range(world):
        err_apply, err_cg, nowned, split_ok = out[rank]
        assert err_apply <= 1e-13, err_apply
        assert err_cg <= 1e-8, err_cg
        assert split_ok
    from tests.problems import hex_case, tet_case

    nnode = hex_case(4, 2)["nnode"] if kind.startswith("hex") else tet_case(4, 2, ncomp=3, perturb=0.1, seed=4)["nnode"]
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


@pytest.mark.parametrize("nranks", [2, 3, 5])
def test_rcb_partition_is_balanced_and_compact(nranks):
    """Recursive coordinate bisection covers every cell once, balances the counts to one cell, and on a shuffled
    numbering keeps the halos far smaller than contiguous cell ranges."""
    from paper_1903_08243_gb300 import dist as mdist
    from tests.problems import hex_case

    case = hex_case(6, 2, shuffle=True)
    ncell = case["cell_vert"].shape[0]
    parts = mdist.rcb_partition(case["coords"], case["cell_vert"], nranks)
    assert np.array_equal(np.sort(np.concatenate(parts)), np.arange(ncell))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1
    halo = lambda ps: sum(mdist.halo_nodes(mdist.build_plan(case["cell_node"], case["nnode"], nranks, r, ps))  # noqa
                          for r in range(nranks))
    assert halo(parts) * 4 < halo(None)


def _sharded_bench_worker(rank, world, port, out):
    """The sharded hex workload of bench.py (its setup and step functions) on a gloo rank, with the oracle as the
    local apply of each part and host tensors (the library kernels need a GPU)."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle

        nx, degrees, forms = 3, (1, 2), ("laplace", "helmholtz")

        class OraclePart:
            def __init__(self, mesh, plan, cells, p, f):
                self.pb = oracle.Problem(oracle.HEX, mesh.coords, mesh.cell_vert[cells], p,
                                         np.ascontiguousarray(plan.local_cell_node[cells]), plan.l2g.size,
                                         bench.FORM_IDS[f], qdeg=p + 1, k2=1.0)

            def apply(self, x, y, accumulate):
                r = torch.from_numpy(self.pb.apply(x.numpy()))
                if accumulate:
                    y += r
                else:
                    y.copy_(r)

        ops = bench.sharded_operators(world, rank, nx, degrees, forms, OraclePart, torch.from_numpy)
        res = []
        for o in ops:
            o["x"][~torch.from_numpy(o["plan"].owned)] = 0.0  # the ghost plane must come from the exchange
            y = bench.sharded_step(o, o["plan"], HostHaloOps())
            res.append((o["name"], o["plan"].l2g.copy(), o["plan"].owned.copy(), y.numpy().copy()))
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_sharded_bench_step_two_ranks():
    """bench.py's sharded hex step on 2 gloo ranks equals the oracle's action on the whole box at every owned
    node, and every node of the box is owned by exactly one rank."""
    import fe_inputs as fi
    import oracle

    world, nx = 2, 3
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_sharded_bench_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    mesh = fi.hex_slab_mesh(nx, nx * world, 0, nx * world)
    for k, (name, _, _, _) in enumerate(out[0]):
        p = int(name[1])
        kind = oracle.LAPLACE if "laplace" in name else oracle.HELMHOLTZ
        cn, nnode = fi.hex_node_map(nx, p, nx * world)
        x = fi.uniform_vector(nnode, seed=1)
        ref = oracle.Problem(oracle.HEX, mesh.coords, mesh.cell_vert, p, cn, nnode, kind, qdeg=p + 1,
                             k2=1.0).apply(x)
        owned = np.zeros(nnode, dtype=int)
        for r in range(world):
            _, l2g, own, y = out[r][k]
            owned[l2g[own]] += 1
            err = np.abs(y[own] - ref[l2g[own]]).max() / np.abs(ref).max()
            assert err <= 1e-13, (name, r, err)
        assert np.all(owned == 1), name
