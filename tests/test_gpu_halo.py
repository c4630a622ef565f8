"""Halo buffers of the cell-partitioned operator on the GPU (mfa_halo_pack / mfa_halo_unpack), and the sharded
hex workload's per-rank parts with both ranks' exchanges carried out in one process (one GPU: the messages are
handed over directly instead of by NCCL), against the oracle's action on the whole box."""
import numpy as np
import pytest

import fe_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1903_08243_gb300 as mfa  # noqa: E402
from paper_1903_08243_gb300 import dist as mdist  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return mfa.Context(0, torch.cuda.current_stream())


@pytest.mark.parametrize("ncomp", [1, 3])
def test_pack_and_unpack(ctx, ncomp):
    rng = np.random.default_rng(ncomp)
    nnode = 5000
    v = rng.standard_normal((nnode, ncomp)) if ncomp > 1 else rng.standard_normal(nnode)
    ids = rng.choice(nnode, size=777, replace=False).astype(np.int32)
    vd, idd = torch.from_numpy(v).cuda(), torch.from_numpy(ids).cuda()
    ops = mdist.LibraryHaloOps(ctx)
    buf = ops.pack(idd, vd)
    ctx.sync()
    assert np.array_equal(buf.cpu().numpy(), v[ids])
    w = torch.zeros_like(vd)
    ops.put(idd, buf, w)
    ops.add(idd, buf, w)
    ctx.sync()
    ref = np.zeros_like(v)
    ref[ids] = 2 * v[ids]
    assert np.array_equal(w.cpu().numpy(), ref)
    # an empty list is a no-op
    ops.put(idd[:0], buf[:0], w)
    ctx.sync()


def test_out_of_range_id_is_reported(ctx):
    v = torch.arange(10, dtype=torch.float64, device="cuda")
    ids = torch.tensor([1, 10, 3], dtype=torch.int32, device="cuda")
    buf = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    mfa.mfa_halo_pack(ctx.h, ids, 1, 10, v, buf)
    with pytest.raises(mfa.MfaError) as e:
        ctx.sync()
    assert e.value.code == mfa.MFA_ERR_RANGE
    assert buf.cpu().tolist() == [1.0, 0.0, 3.0]  # the bad entry packs 0; the others are moved
    mfa.mfa_halo_unpack(ctx.h, ids, 1, 10, buf, v, True)
    with pytest.raises(mfa.MfaError):
        ctx.sync()
    assert v.cpu().tolist()[1] == 2.0 and v.cpu().tolist()[3] == 6.0
    ctx.sync()  # the flag was cleared and the context stays usable


@pytest.mark.parametrize("p", [1, 3, 6])
def test_two_slab_ranks_in_one_process(ctx, p):
    """bench.py's sharded setup for ranks 0 and 1 of 2, the parts applied by the library, the import and reverse
    exchanges packed and unpacked by the library kernels: the owned entries equal the oracle's action on the
    whole box (a single domain), and every node is owned once."""
    import bench

    nx, world = 3, 2
    keep = []

    class Part:
        def __init__(self, mesh, plan, cells, p_, f):
            m = mfa.Mesh(ctx, mfa.MFA_CELL_HEX8, mesh.coords, np.ascontiguousarray(mesh.cell_vert[cells]))
            sp = mfa.Space(m, p_, 1, np.ascontiguousarray(plan.local_cell_node[cells]), plan.l2g.size)
            self.form = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, k2=1.0)
            keep.append((m, sp))

        def apply(self, x, y, accumulate):
            mfa.mfa_apply(ctx.h, self.form.h, x, y, accumulate)

    ranks = [bench.sharded_operators(world, r, nx, [p], ["helmholtz"], Part, lambda a: torch.from_numpy(a).cuda())[0]
             for r in range(world)]
    halo = mdist.LibraryHaloOps(ctx)
    plans = [mdist.device_plan(o["plan"], "cuda") for o in ranks]
    for o in ranks:
        o["x"][~torch.from_numpy(o["plan"].owned).cuda()] = 0.0  # ghosts come from the import
    # import: rank 0 sends its top plane, rank 1 receives it as its ghost plane
    buf = halo.pack(plans[0].send_import[1], ranks[0]["x"])
    halo.put(plans[1].recv_import[0], buf, ranks[1]["x"])
    for o in ranks:
        b, i = o["parts"]["boundary"], o["parts"]["interior"]
        b.apply(o["x"], o["y"], False)
        i.apply(o["x"], o["y"], True)
    # reverse: rank 1's partial sums at its ghost plane are added into rank 0's owned plane
    buf = halo.pack(plans[1].send_reverse[0], ranks[1]["y"])
    halo.add(plans[0].recv_reverse[1], buf, ranks[0]["y"])
    ctx.sync()
    mesh = fi.hex_slab_mesh(nx, nx * world, 0, nx * world)
    cn, nnode = fi.hex_node_map(nx, p, nx * world)
    x = fi.uniform_vector(nnode, seed=1)
    ref = oracle.Problem(oracle.HEX, mesh.coords, mesh.cell_vert, p, cn, nnode, oracle.HELMHOLTZ, qdeg=p + 1,
                         k2=1.0).apply(x)
    owned = np.zeros(nnode, dtype=int)
    for o in ranks:
        pl = o["plan"]
        y = o["y"].cpu().numpy()
        owned[pl.l2g[pl.owned]] += 1
        err = np.abs(y[pl.owned] - ref[pl.l2g[pl.owned]]).max() / np.abs(ref).max()
        assert err <= 1e-13, err
    assert np.all(owned == 1)
