"""Cell-partitioned operator action across ranks: one halo exchange per apply.

Global assembly (Section 2.2 of arXiv 1903.08243) sums cell contributions
into shared dofs.  Partitioning the cells over R ranks leaves each node
either interior to one rank or shared by several.  Every node is owned by
the lowest rank that touches it; the other ranks that touch it hold it as a
ghost.  One distributed apply is then

  1. import: owners send the current x at every ghost node to the ranks that
     hold the ghost (so each rank sees x on all nodes of its cells),
  2. local apply on the rank's cells (the GPU kernels in production),
  3. reverse add: each rank sends its partial sums at ghost nodes to the owner,
     which adds them, so each owned entry of y is the full global sum.

Scalars of Krylov methods are sums over owned entries, all-reduced.  The
exchange uses torch.distributed point-to-point messages between neighbouring
ranks (NCCL between GPUs), posted as one group per exchange.  Moving values
between a node vector and a message buffer is the job of a halo-ops object:
on the GPU, LibraryHaloOps runs the library's kernels (mfa_halo_pack /
mfa_halo_unpack) on the context stream.

The overlapped apply splits a rank's cells into boundary cells (touching a
node shared with another rank) and interior cells (touching none): after the
import, the boundary cells are applied first, which completes the partial sums
at every shared node; the reverse exchange is then in flight while the
interior cells are applied, since those touch no shared node.  In production
each part is its own form (two meshes over the rank's node numbering, the
second applied with accumulate).
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class HaloPlan:
    rank: int
    nranks: int
    cells: np.ndarray            # global ids of this rank's cells
    local_cell_node: np.ndarray  # [ncell_local][nloc] in local node ids
    l2g: np.ndarray              # local node -> global node
    owned: np.ndarray            # bool per local node
    # per neighbour rank: local ids this rank sends / receives
    send_import: dict = field(default_factory=dict)  # owned nodes whose x a neighbour needs
    recv_import: dict = field(default_factory=dict)  # ghost nodes whose x comes from the owner
    send_reverse: dict = field(default_factory=dict)  # ghost nodes whose partial y goes to the owner
    recv_reverse: dict = field(default_factory=dict)  # owned nodes receiving partial y from a neighbour
    boundary_cells: np.ndarray = None  # local cell indices touching a node shared with another rank
    interior_cells: np.ndarray = None  # local cell indices touching no shared node


def contiguous_partition(ncell, nranks):
    """Cell ranges [start, end) per rank (z-slabs on a lexicographic structured mesh)."""
    bounds = np.linspace(0, ncell, nranks + 1).round().astype(np.int64)
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(nranks)]


def rcb_partition(coords, cell_vert, nranks):
    """Recursive coordinate bisection of the cells by their centroids: each split cuts the longest extent of
    the current set at the cell count proportional to the ranks on either side.  Compact parts whatever the
    cell numbering (shuffled or unstructured meshes), so halos stay small.  Returns sorted cell ids per rank."""
    cent = np.asarray(coords)[np.asarray(cell_vert)].mean(axis=1)
    out = []

    def split(ids, k):
        if k == 1:
            out.append(np.sort(ids))
            return
        ext = cent[ids].max(axis=0) - cent[ids].min(axis=0)
        axis = int(np.argmax(ext))
        order = ids[np.argsort(cent[ids, axis], kind="stable")]
        k0 = k // 2
        cut = int(round(len(ids) * k0 / k))
        split(order[:cut], k0)
        split(order[cut:], k - k0)

    split(np.arange(len(cent), dtype=np.int64), nranks)
    return out


def _part_cells(part):
    """A part given as a (start, end) range or as an array of cell ids."""
    if isinstance(part, tuple):
        return np.arange(part[0], part[1], dtype=np.int64)
    return np.asarray(part, dtype=np.int64)


def build_plan(cell_node, nnode, nranks, rank, parts=None):
    """Halo plan of `rank`; every rank computes the same global ownership.  parts: per rank a (start, end) range
    or an array of cell ids (contiguous_partition, rcb_partition); default contiguous ranges."""
    ncell = cell_node.shape[0]
    parts = parts or contiguous_partition(ncell, nranks)
    touch_min = np.full(nnode, nranks, dtype=np.int64)  # owner = lowest rank touching the node
    touched_by = [None] * nranks
    for r, part in enumerate(parts):
        nodes = np.unique(cell_node[_part_cells(part)])
        touched_by[r] = nodes
        touch_min[nodes] = np.minimum(touch_min[nodes], r)
    cells = _part_cells(parts[rank])
    l2g, local = np.unique(cell_node[cells], return_inverse=True)
    plan = HaloPlan(rank=rank, nranks=nranks, cells=cells,
                    local_cell_node=local.reshape(len(cells), -1).astype(np.int32), l2g=l2g,
                    owned=touch_min[l2g] == rank)
    g2l = {int(g): i for i, g in enumerate(l2g)}
    for other in range(nranks):
        if other == rank:
            continue
        shared = np.intersect1d(l2g, touched_by[other], assume_unique=True)
        if shared.size == 0:
            continue
        mine = shared[touch_min[shared] == rank]       # I own, `other` holds as ghost
        theirs = shared[touch_min[shared] == other]    # `other` owns, I hold as ghost
        if mine.size:
            ids = np.array([g2l[int(g)] for g in mine], dtype=np.int64)
            plan.send_import[other] = ids
            plan.recv_reverse[other] = ids
        if theirs.size:
            ids = np.array([g2l[int(g)] for g in theirs], dtype=np.int64)
            plan.recv_import[other] = ids
            plan.send_reverse[other] = ids
    shared = np.zeros(l2g.size, dtype=bool)
    for ids in list(plan.send_import.values()) + list(plan.recv_import.values()):
        shared[ids] = True
    on_boundary = shared[plan.local_cell_node].any(axis=1)
    plan.boundary_cells = np.flatnonzero(on_boundary)
    plan.interior_cells = np.flatnonzero(~on_boundary)
    return plan


def slab_plan(nx, nz, p, nranks, rank):
    """Halo plan of a z-slab partition of the structured Q_p hex mesh of nx * nx * (nz * nranks) cells, computed
    from the lattice instead of from the global map (build_plan gives the same plan for contiguous_partition).

    Rank r owns cell layers [r nz, (r + 1) nz); its local nodes are the (nx p + 1)^2 (nz p + 1) lattice nodes of
    its slab, numbered lexicographically (the map of fe_inputs.hex_node_map(nx, p, nz)), which are consecutive
    global nodes.  The node plane shared with rank r - 1 (local plane 0) is owned by r - 1, the lowest rank that
    touches it: a ghost here.  The plane shared with rank r + 1 (local plane nz p) is owned here.  Boundary cells
    are the cell layers that touch a shared plane."""
    import fe_inputs as fi

    m = nx * p + 1
    plane = m * m
    cell_node, nlocal = fi.hex_node_map(nx, p, nz)
    cells_per_rank = nx * nx * nz
    plan = HaloPlan(rank=rank, nranks=nranks,
                    cells=rank * cells_per_rank + np.arange(cells_per_rank, dtype=np.int64),
                    local_cell_node=cell_node, l2g=rank * nz * p * plane + np.arange(nlocal, dtype=np.int64),
                    owned=np.ones(nlocal, dtype=bool))
    bottom = np.arange(plane, dtype=np.int64)
    top = nz * p * plane + np.arange(plane, dtype=np.int64)
    layer = np.arange(cells_per_rank) // (nx * nx)
    on_boundary = np.zeros(cells_per_rank, dtype=bool)
    if rank > 0:
        plan.owned[bottom] = False
        plan.recv_import[rank - 1] = bottom
        plan.send_reverse[rank - 1] = bottom
        on_boundary |= layer == 0
    if rank < nranks - 1:
        plan.send_import[rank + 1] = top
        plan.recv_reverse[rank + 1] = top
        on_boundary |= layer == nz - 1
    plan.boundary_cells = np.flatnonzero(on_boundary)
    plan.interior_cells = np.flatnonzero(~on_boundary)
    return plan


class LibraryHaloOps:
    """Halo buffers moved by the library's kernels on the context stream (device tensors).

    pack(ids, v) returns the buffer v[ids]; put(ids, buf, v) sets v[ids] = buf; add(ids, buf, v) adds buf into
    v[ids].  ids: int32 device tensors (see device_plan); v: float64 [nnode] or [nnode][ncomp]."""

    def __init__(self, ctx):
        self.ctx = ctx

    @staticmethod
    def _shape(v):
        return (v.shape[0], 1 if v.dim() == 1 else int(v.shape[1]))

    def pack(self, ids, v):
        import torch

        from . import mfa_halo_pack

        nnode, nc = self._shape(v)
        buf = torch.empty((ids.numel(),) + tuple(v.shape[1:]), dtype=v.dtype, device=v.device)
        mfa_halo_pack(self.ctx.h, ids, nc, nnode, v, buf)
        return buf

    def put(self, ids, buf, v):
        from . import mfa_halo_unpack

        nnode, nc = self._shape(v)
        mfa_halo_unpack(self.ctx.h, ids, nc, nnode, buf, v, False)

    def add(self, ids, buf, v):
        from . import mfa_halo_unpack

        nnode, nc = self._shape(v)
        mfa_halo_unpack(self.ctx.h, ids, nc, nnode, buf, v, True)


def device_plan(plan, device):
    """A copy of the plan whose exchange lists are int32 tensors on `device` (uploaded once, reused by every
    exchange)."""
    import copy

    import torch

    out = copy.copy(plan)
    for name in ("send_import", "recv_import", "send_reverse", "recv_reverse"):
        setattr(out, name, {peer: torch.as_tensor(np.asarray(ids, dtype=np.int32), device=device)
                            for peer, ids in getattr(plan, name).items()})
    return out


def _start_exchange(send, recv, values, ops):
    """Post the point-to-point messages of one exchange as one group: the packed values[ids] to each peer, and a
    buffer per peer to receive into."""
    import torch
    import torch.distributed as dist

    p2p, bufs = [], {}
    for peer, ids in recv.items():
        buf = torch.empty((len(ids),) + tuple(values.shape[1:]), dtype=values.dtype, device=values.device)
        bufs[peer] = buf
        p2p.append(dist.P2POp(dist.irecv, buf, peer))
    for peer, ids in send.items():
        p2p.append(dist.P2POp(dist.isend, ops.pack(ids, values), peer))
    reqs = dist.batch_isend_irecv(p2p) if p2p else []
    return reqs, bufs


def _finish_exchange(recv, values, combine, pending):
    reqs, bufs = pending
    for r in reqs:
        r.wait()
    for peer, ids in recv.items():
        combine(ids, bufs[peer], values)


def _exchange(send, recv, values, combine, ops):
    """Point-to-point exchange: send values[ids] to each peer, combine received data at ids."""
    _finish_exchange(recv, values, combine, _start_exchange(send, recv, values, ops))


def import_ghosts(plan, x_local, ops):
    """x at ghost nodes <- owner's value."""
    _exchange(plan.send_import, plan.recv_import, x_local, ops.put, ops)


def reverse_add(plan, y_local, ops, refresh=True):
    """Owner's y += each neighbour's partial sums at its ghost copies; with refresh the ghosts then hold the
    full value too."""
    _exchange(plan.send_reverse, plan.recv_reverse, y_local, ops.add, ops)
    if refresh:
        import_ghosts(plan, y_local, ops)  # make ghost copies consistent with the owner


def distributed_apply(plan, local_apply, x_local, ops):
    """y_local = (A x)_local on every local node (owned and ghost), x_local holding owned values."""
    import_ghosts(plan, x_local, ops)
    y = local_apply(x_local)
    reverse_add(plan, y, ops)
    return y


def distributed_apply_overlapped(plan, apply_boundary, apply_interior, x_local, ops, y=None, refresh=True):
    """distributed_apply with the reverse exchange in flight during the interior cells.

    apply_boundary(x, y) and apply_interior(x, y) apply the rank's boundary and interior cells
    (plan.boundary_cells, plan.interior_cells): the first overwrites y, the second adds into it (y is allocated
    by apply_boundary's caller when None: apply_boundary(x, None) returns it).  Without refresh the ghost
    entries of y keep this rank's partial sums (the owned entries are complete either way)."""
    import_ghosts(plan, x_local, ops)
    y = apply_boundary(x_local, y)  # every shared node's partial sum is now final on this rank
    pending = _start_exchange(plan.send_reverse, plan.recv_reverse, y, ops)  # partial sums at ghosts -> owners
    apply_interior(x_local, y)  # touches no shared node: cannot race with the messages
    _finish_exchange(plan.recv_reverse, y, ops.add, pending)
    if refresh:
        import_ghosts(plan, y, ops)  # ghost copies take the owners' full sums
    return y


def halo_nodes(plan):
    """Ghost nodes of the plan (nodes this rank touches and another rank owns)."""
    return int((~plan.owned).sum())


def owned_dot(plan, a, b):
    import torch
    import torch.distributed as dist

    mask = torch.as_tensor(plan.owned, device=a.device)
    s = (a[mask] * b[mask]).sum().reshape(1)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(s.item())


def distributed_cg(plan, local_apply, b_local, x_local, ops, diag_local=None, rtol=1e-8, maxit=1000,
                   overlapped=None):
    """Jacobi-preconditioned CG over the partitioned operator (reference logic for N > 1).

    overlapped: (apply_boundary, apply_interior) to use distributed_apply_overlapped instead."""
    def dapply(v):
        if overlapped is not None:
            return distributed_apply_overlapped(plan, overlapped[0], overlapped[1], v, ops)
        return distributed_apply(plan, local_apply, v, ops)

    r = b_local - dapply(x_local.clone())
    dinv = None if diag_local is None else 1.0 / diag_local
    z = r if dinv is None else dinv * r
    p = z.clone()
    rz = owned_dot(plan, r, z)
    bnorm = owned_dot(plan, b_local, b_local) ** 0.5
    it, res = 0, owned_dot(plan, r, r) ** 0.5 / bnorm
    while res > rtol and it < maxit:
        q = dapply(p.clone())
        alpha = rz / owned_dot(plan, p, q)
        x_local += alpha * p
        r -= alpha * q
        it += 1
        res = owned_dot(plan, r, r) ** 0.5 / bnorm
        if res <= rtol:
            break
        z = r if dinv is None else dinv * r
        rz_new = owned_dot(plan, r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x_local, it, res
