#!/usr/bin/env python
"""Benchmark of the matrix-free finite element operator action on GB300.

Default workload: Laplacian and Helmholtz (k^2 = 1) actions of scalar Q_p,
p = 1..6, on a 64^3 hexahedral mesh with vertices perturbed by up to 0.1h,
p+1 Gauss points per direction, sum-factorised, FP64, input uniform in
[-1, 1) (the Section 4 operator-action experiment on the hex mesh).  One
step applies all 12 operators once; the metric is the operator action rate
in GDoF/s (global dofs processed per second, summed over the operators).

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample (a box of cells cut from the same mesh) per operator.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fe_inputs as fi  # noqa: E402

# FP64 pipe of GB300: 152 SMs x 2 DFMA lanes/clk x 2 flop x 2070 MHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# DRAM traffic per launch of the dominant kernel from one ncu capture, keyed by the
# sha1 (first 12 hex digits) of the kernel's source file and the operator, so that
# it is reported only while that source is unchanged.  Even-odd kernel (hex_eo.cuh),
# Q6 Helmholtz: the 32^3 capture (869.22 MB per launch) scaled by the cell count to
# the 64^3 launch (profiles/eo_apply_q6_helmholtz_hex32.md).
NCU_TRAFFIC = {("7855a4e73280", "Q6 helmholtz"): 8 * 868.7e6}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mfa", "reference"], default="mfa")
    ap.add_argument("--workload", choices=["hex", "hex-vector", "tet-pk", "planar", "tet-p1-mass", "tet-p2", "batched",
                                           "pcg", "pcg-elasticity"],
                    default="hex",
                    help="hex: 64^3 Q1-Q6 Laplace+Helmholtz; tet-p1-mass: 8^3x6 P1 mass; "
                         "tet-p2: 48^3x6 vector P2 elasticity + neo-Hookean residual; "
                         "batched: 64 hex Helmholtz operators (degrees 1-8, 8^3-48^3) in one graph; "
                         "pcg: Q4 64^3 Helmholtz solves to 1e-8, FP64 Jacobi-PCG vs mixed-precision FCG")
    ap.add_argument("--nrhs", type=int, default=2, help="pcg: right-hand sides timed")
    ap.add_argument("--inner", type=int, default=16, help="pcg: inner FP32 Jacobi-PCG steps per outer step")
    ap.add_argument("--inner-precision", choices=["fp32", "bf16", "fp64"], default="fp32")
    ap.add_argument("--train-rhs", type=int, default=3)
    ap.add_argument("--train-steps", type=int, default=800)
    ap.add_argument("--train-lr", type=float, default=2e-3)
    ap.add_argument("--train-data", choices=["grf", "white", "mixed"], default="white")
    ap.add_argument("--lanczos", type=int, default=300, help="pcg: PCG steps of the spectrum estimate")
    ap.add_argument("--precision", choices=["fp64", "fp32", "bf16"], default=None,
                    help="arithmetic (hex and batched workloads; default fp64 for hex, fp32 for batched)")
    ap.add_argument("--nops", type=int, default=64)
    ap.add_argument("--nx", type=int, default=None)
    ap.add_argument("--graph", action="store_true", help="replay each step from a captured CUDA graph")
    ap.add_argument("--degrees", default=None, help="hex: 1,2,3,4,5,6; hex-vector: 1,2,3,4")
    ap.add_argument("--forms", default=None,
                    help="hex: laplace,helmholtz; hex-vector: elasticity,hyper_res,hyper_jac "
                         "(neo-Hookean residual, St Venant-Kirchhoff Jacobian action)")
    ap.add_argument("--scatter", choices=["atomic", "colour", "warp"], default="atomic",
                    help="scatter at form creation (the autotuner may change it)")
    ap.add_argument("--rule", choices=["auto", "symmetric"], default="auto",
                    help="simplices: the cheapest exact rule where the integrand is a polynomial (auto), or Table 2's "
                         "symmetric rules whatever the integrand (symmetric; changes the neo-Hookean result)")
    ap.add_argument("--geometry", choices=["stored", "onthefly"], default="stored",
                    help="hex FP64: geometric factors stored at setup, or recomputed at every point from the vertices")
    ap.add_argument("--order", choices=["lex", "shuffled", "rcm"], default="lex",
                    help="cell and node numbering: generator (lexicographic), seeded random permutation, or the "
                         "random permutation renumbered by the library's reverse Cuthill-McKee")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep each form's default launch configuration instead of timing all of them")
    ap.add_argument("--parallelism", choices=["auto", "sharded", "replicas"], default="auto",
                    help="N > 1: the hex workload shards a box of N nx^3 z-slabs over the ranks (auto), the others "
                         "run a replica per rank")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    return ap.parse_args()


FORM_IDS = {"mass": 0, "laplace": 1, "helmholtz": 2, "elasticity": 3, "hyper_res": 4, "hyper_jac": 5}


def workload_name(args):
    return (_workload_name(args) + ("" if args.order == "lex" else "-order-" + args.order) +
            ("-geometry-onthefly" if args.geometry == "onthefly" else "") +
            ("-rule-symmetric" if args.rule == "symmetric" else ""))


def renumber(args, cell_vert, cell_node, nnode, nvert, vectors):
    """The maps and node vectors in the numbering `args.order` asks for.  `vectors`: node-major arrays
    (nnode * ncomp values each) that follow the node permutation."""
    if args.order == "lex":
        return cell_vert, cell_node, vectors
    cv, cn, perm = fi.shuffle_mesh(cell_vert, cell_node, nnode, seed=7)
    if args.order == "rcm":
        from paper_1903_08243_gb300 import build as libbuild

        libbuild.build()
        import paper_1903_08243_gb300 as mfa

        order, perm2 = mfa.mfa_order_rcm(cv, cn, nnode, nvert=nvert)
        cv, cn = mfa.apply_order(cv, cn, order, perm2)
        perm = perm2[perm]
    out = []
    for v in vectors:
        if v is None:
            out.append(None)
            continue
        w = np.empty_like(v.reshape(nnode, -1))
        w[perm] = v.reshape(nnode, -1)
        out.append(w.ravel())
    return cv, cn, out


def _workload_name(args):
    if args.workload in ("hex", "hex-vector"):
        return "hex%d^3-perturbed0.1h-Q%s-%s%s-%s" % (args.nx, args.degrees.replace(",", ""),
                                                      "vector-" if args.workload == "hex-vector" else "",
                                                      args.forms.replace(",", "+"),
                                                      args.precision if args.workload == "hex" else "fp64")
    if args.workload == "tet-p1-mass":
        return "tet-kuhn%d^3x6-P1-mass-fp64" % args.nx
    if args.workload == "tet-pk":
        return "tet-kuhn%d^3x6-P%s-%s-fp64" % (args.nx, args.degrees.replace(",", ""), args.forms.replace(",", "+"))
    if args.workload == "planar":
        return "quad%d^2+tri%d^2x2-p%s-%s-fp64" % (args.nx, args.nx // 2, args.degrees.replace(",", ""),
                                                    args.forms.replace(",", "+"))
    return "tet-kuhn%d^3x6-P2vec-elasticity+neohookean-residual-fp64" % args.nx


def build_cases(args):
    """Operators of one step.  Each case holds the seeded inputs shared by the GPU and the oracle."""
    if args.nx is None:
        args.nx = {"hex": 64, "hex-vector": 48, "tet-pk": 16, "planar": 512, "tet-p1-mass": 8,
                   "tet-p2": 48}[args.workload]
    cases = []
    if args.workload == "hex-vector":
        mesh = fi.hex_box_mesh(args.nx, perturb=0.1, seed=1)
        laws = {"elasticity": 0, "laplace": 0, "hyper_res": 1, "hyper_jac": 0}
        lawname = {"elasticity": "", "laplace": "", "hyper_res": " neo-Hookean", "hyper_jac": " SVK"}
        for p in [int(p) for p in args.degrees.split(",")]:
            cell_node, nnode = fi.hex_node_map(args.nx, p)
            m1 = args.nx * p + 1
            v = np.arange(nnode)
            grid = np.stack([v % m1, (v // m1) % m1, v // (m1 * m1)], axis=1) / (m1 - 1)
            u = fi.sinusoid_displacement(grid, seed=2).ravel()  # smooth field on the node grid
            xr = fi.uniform_vector(3 * nnode, seed=1)
            cv, cell_node, (u, xr) = renumber(args, mesh.cell_vert, cell_node, nnode, mesh.nvert, [u, xr])
            for f in args.forms.split(","):
                kw = dict(lam=1.0, mu=1.0, law=laws[f])
                cases.append(dict(name="Q%d %s%s" % (p, f, lawname[f]), cell_type=8, mesh=mesh, p=p, ncomp=3, form=f,
                                  cell_vert=cv, cell_node=cell_node, nnode=nnode, x=u if f == "hyper_res" else xr,
                                  coef=u if f == "hyper_jac" else None, kw=kw, okw=kw, qdeg=p + 1))
    elif args.workload == "hex":
        mesh = fi.hex_box_mesh(args.nx, perturb=0.1, seed=1)
        for p in [int(p) for p in args.degrees.split(",")]:
            cell_node, nnode = fi.hex_node_map(args.nx, p)
            x = fi.uniform_vector(nnode, seed=1)
            cv, cell_node, (x,) = renumber(args, mesh.cell_vert, cell_node, nnode, mesh.nvert, [x])
            for f in args.forms.split(","):
                cases.append(dict(name="Q%d %s" % (p, f), cell_type=8, mesh=mesh, p=p, ncomp=1, form=f,
                                  cell_vert=cv, cell_node=cell_node, nnode=nnode, x=x, kw=dict(k2=1.0),
                                  okw=dict(k2=1.0), qdeg=p + 1))
    elif args.workload == "planar":
        for cell in ("quad", "tri"):
            mesh = fi.quad_mesh(args.nx, perturb=0.1, seed=1) if cell == "quad" else fi.tri_mesh(args.nx // 2,
                                                                                                 perturb=0.1, seed=1)
            for p in [int(p) for p in args.degrees.split(",")]:
                if cell == "quad":
                    cn, nnode = fi.quad_node_map(args.nx, p)
                    m1 = args.nx * p + 1
                    v = np.arange(nnode)
                    nodes = np.stack([v % m1, v // m1, np.zeros(nnode)], axis=1) / (m1 - 1)  # the node grid
                else:
                    cn, nnode, node_coords = fi.tri_node_map(mesh.cell_vert, mesh.nvert, p)
                    nodes = node_coords(mesh.coords)
                for f in args.forms.split(","):
                    nc = 2 if f in ("elasticity", "hyper_res", "hyper_jac") else 1
                    if nc == 2:
                        x = fi.sinusoid_displacement(nodes, seed=2)[:, :2].ravel()
                        kw = dict(lam=1.0, mu=1.0, law=1)
                    else:
                        x = fi.uniform_vector(nnode, seed=0)
                        kw = dict(k2=1.0)
                    ct = 40 if cell == "quad" else 3
                    qd = p + 1 if cell == "quad" else (max(4, 2 * p) if f.startswith("hyper") else 2 * p)
                    cases.append(dict(name="%s %s%d %s" % (cell, "Q" if cell == "quad" else "P", p, f), cell_type=ct,
                                      mesh=mesh, p=p, ncomp=nc, form=f, cell_vert=mesh.cell_vert, cell_node=cn,
                                      nnode=nnode, x=x, kw=kw, okw=kw, qdeg=qd))
    elif args.workload == "tet-pk":
        mesh = fi.kuhn_tet_mesh(args.nx)
        for p in [int(p) for p in args.degrees.split(",")]:
            cn, nnode, node_coords = fi.pk_node_map(mesh.cell_vert, mesh.nvert, p)
            nodes = node_coords(mesh.coords)
            for f in args.forms.split(","):
                nc = 3 if f in ("elasticity", "hyper_res", "hyper_jac") else 1
                if nc == 3:
                    x = fi.sinusoid_displacement(nodes, seed=2).ravel()
                    kw = dict(lam=1.0, mu=1.0, law=1)
                else:
                    x = fi.uniform_vector(nnode, seed=0)
                    kw = dict(k2=1.0)
                cv, cnr, (x,) = renumber(args, mesh.cell_vert, cn, nnode, mesh.nvert, [x])
                cases.append(dict(name="P%d %s" % (p, f), cell_type=4, mesh=mesh, p=p, ncomp=nc, form=f,
                                  cell_vert=cv, cell_node=cnr, nnode=nnode, x=x, kw=kw, okw=kw,
                                  qdeg=(max(4, 2 * p) if f.startswith("hyper") else 2 * p)))
    elif args.workload == "tet-p1-mass":
        mesh = fi.kuhn_tet_mesh(args.nx)
        x = fi.uniform_vector(mesh.nvert, seed=0)
        cv, cn, (x,) = renumber(args, mesh.cell_vert, mesh.cell_vert, mesh.nvert, mesh.nvert, [x])
        cases.append(dict(name="P1 mass", cell_type=4, mesh=mesh, p=1, ncomp=1, form="mass", cell_vert=cv,
                          cell_node=cn, nnode=mesh.nvert, x=x, kw={}, okw={}, qdeg=2))
    else:
        mesh = fi.kuhn_tet_mesh(args.nx)
        cn, nnode, edges = fi.p2_node_map(mesh.cell_vert, mesh.nvert)
        u = fi.sinusoid_displacement(fi.p2_node_coords(mesh.coords, edges), seed=2).ravel()
        cv, cn, (u,) = renumber(args, mesh.cell_vert, cn, nnode, mesh.nvert, [u])
        cases.append(dict(name="P2 elasticity", cell_type=4, mesh=mesh, p=2, ncomp=3, form="elasticity",
                          cell_vert=cv, cell_node=cn, nnode=nnode, x=u, kw=dict(lam=1.0, mu=1.0),
                          okw=dict(lam=1.0, mu=1.0), qdeg=4))
        cases.append(dict(name="P2 neo-Hookean residual", cell_type=4, mesh=mesh, p=2, ncomp=3, form="hyper_res",
                          cell_vert=cv, cell_node=cn, nnode=nnode, x=u, kw=dict(lam=1.0, mu=1.0, law=1),
                          okw=dict(lam=1.0, mu=1.0, law=1), qdeg=4))
    for c in cases:
        c["ndof"] = c["nnode"] * c["ncomp"]
        if getattr(args, "rule", "auto") == "symmetric" and c["cell_type"] in (3, 4):
            c["okw"] = dict(c["okw"], rule="symmetric")  # the oracle legs integrate with the same rules
    return cases


# launch-configuration variant -> (header holding the kernel, kernel name)
VARIANT_KERNELS = {1: ("hex_kernels.cuh", "hex_apply_kernel"), 2: ("hex_eo.cuh", "eo_apply_kernel"),
                   3: ("hex_lines.cuh", "line_apply_kernel"), 4: ("hex_lines.cuh", "line_apply_kernel")}


def kernel_hash(name="hex_kernels.cuh"):
    src = os.path.join(ROOT, "paper_1903_08243_gb300", "csrc", name)
    return hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_link_gbs(nbytes=512 << 20, reps=3):
    """The host link as the end-to-end leg meets it: one pinned host->device copy, one device->host copy, then
    both at once on two streams, each timed with CUDA events on its own stream (median of `reps`). Context for
    the e2e figure only: these copies are plain cudaMemcpyAsync calls made by torch, not part of the library."""
    import torch

    n = nbytes // 8
    h_in = torch.empty(n, dtype=torch.float64).pin_memory()
    h_out = torch.empty(n, dtype=torch.float64).pin_memory()
    d_in = torch.empty(n, dtype=torch.float64, device="cuda")
    d_out = torch.zeros(n, dtype=torch.float64, device="cuda")
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(which):
        t = {}
        ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in which}
        torch.cuda.synchronize()
        if "h2d" in which:
            with torch.cuda.stream(s_in):
                ev["h2d"][0].record(s_in)
                d_in.copy_(h_in, non_blocking=True)
                ev["h2d"][1].record(s_in)
        if "d2h" in which:
            with torch.cuda.stream(s_out):
                ev["d2h"][0].record(s_out)
                h_out.copy_(d_out, non_blocking=True)
                ev["d2h"][1].record(s_out)
        torch.cuda.synchronize()
        for k in which:
            t[k] = ev[k][0].elapsed_time(ev[k][1]) / 1e3
        return t

    timed(("h2d", "d2h"))  # first touch of the pinned pages and the streams
    alone = {"h2d": [], "d2h": []}
    both = {"h2d": [], "d2h": []}
    for _ in range(reps):
        for k in ("h2d", "d2h"):
            alone[k].append(timed((k,))[k])
        t = timed(("h2d", "d2h"))
        for k in t:
            both[k].append(t[k])
    gbs = lambda ts: nbytes / statistics.median(ts) / 1e9  # noqa: E731
    return {"h2d_gbs": gbs(alone["h2d"]), "d2h_gbs": gbs(alone["d2h"]),
            "h2d_gbs_concurrent": gbs(both["h2d"]), "d2h_gbs_concurrent": gbs(both["d2h"]),
            "bytes_per_copy": nbytes, "source": "pinned torch tensors, one cudaMemcpyAsync per direction, CUDA events"}


# ------------------------------------------------------------------ CPU oracle (baseline / reference arm)

def sub_mesh(case, ncell_sample):
    """The first cells of the mesh (a slab of boxes), with compact node numbering."""
    cells = np.arange(min(ncell_sample, case["mesh"].ncell))
    cv, cn = case["cell_vert"][cells], case["cell_node"][cells]
    nodes, inv = np.unique(cn, return_inverse=True)
    return cv, inv.reshape(cn.shape).astype(np.int32), nodes, cells.size


# Cells per oracle sample: about 1-2.5 s of oracle work per operator for the
# baseline, about 0.1 s per operator and step for the reference arm.
SAMPLE_CPU_LEG = {("quad", 1): 200000, ("quad", 2): 100000, ("quad", 3): 50000, ("quad", 4): 25000,
                   ("tri", 1): 100000, ("tri", 2): 50000, ("tri", 3): 20000, ("tri", 4): 10000, ("tet", 3): 6000, ("tet", 4): 1500, ("tet", 5): 400, ("tet", 6): 150,("hex", 1): 262144, ("hex", 2): 64000, ("hex", 3): 21952, ("hex", 4): 8000, ("hex", 5): 2744,
                   ("hex", 6): 1728, ("hex", 7): 512, ("hex", 8): 216, ("tet", 1): 3072, ("tet", 2): 200000,
                   ("hexv", 1): 110592, ("hexv", 2): 24000, ("hexv", 3): 4000, ("hexv", 4): 1000, ("hexv", 5): 250,
                   ("hexv", 6): 100}
SAMPLE_STEP = {("quad", 1): 20000, ("quad", 2): 8000, ("quad", 3): 3000, ("quad", 4): 1500, ("tri", 1): 10000,
               ("tri", 2): 4000, ("tri", 3): 1500, ("tri", 4): 700, ("tet", 3): 400, ("tet", 4): 100, ("tet", 5): 30, ("tet", 6): 12,("hex", 1): 13824, ("hex", 2): 2744, ("hex", 3): 1000, ("hex", 4): 512, ("hex", 5): 216,
               ("hex", 6): 125, ("hex", 7): 64, ("hex", 8): 27, ("tet", 1): 3072, ("tet", 2): 6000,
               ("hexv", 1): 8000, ("hexv", 2): 1500, ("hexv", 3): 250, ("hexv", 4): 64, ("hexv", 5): 16,
               ("hexv", 6): 8}


def oracle_rate(cases, repeats=1, samples=SAMPLE_STEP):
    """Extrapolated full-mesh oracle time per operator: the oracle timed on the first n/2 and the first n cells of
    the mesh; full time = fixed part (its per-call setup: rules and basis tables) + per-cell slope x cells."""
    import oracle

    out = []
    for c in cases:
        ncell = c["mesh"].ncell
        key = ({3: "tri", 4: "tet", 40: "quad"}.get(c["cell_type"]) or ("hexv" if c["ncomp"] == 3 else "hex"), c["p"])
        n_big = min(samples.get(key, 64), ncell)
        times = []
        for n in sorted({max(1, n_big // 2), n_big}):
            cv, cn, nodes, nsub = sub_mesh(c, n)
            coef = None if c.get("coef") is None else c["coef"].reshape(-1, c["ncomp"])[nodes].ravel()
            xs = c["x"].reshape(-1, c["ncomp"])[nodes].ravel()
            pb = oracle.Problem(c["cell_type"], c["mesh"].coords, cv, c["p"], cn, nodes.size, FORM_IDS[c["form"]],
                                ncomp=c["ncomp"], qdeg=c["qdeg"], ucoef=coef, **c["okw"])
            best = None
            for _ in range(repeats):
                t0 = time.perf_counter()
                pb.apply(xs)
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            times.append((nsub, best))
        if len(times) == 2 and times[1][0] > times[0][0]:
            (n1, t1), (n2, t2) = times
            slope = max(t2 - t1, 0.0) / (n2 - n1)
            fixed = max(t1 - slope * n1, 0.0)
        else:
            (n2, t2), fixed, slope = times[-1], 0.0, times[-1][1] / times[-1][0]
        out.append(dict(name=c["name"], sample_cells=n2, sample_s=t2, full_s=fixed + slope * ncell, ndof=c["ndof"],
                        fixed_s=fixed))
    return out


def _oracle_chunk_apply(task):
    """One worker of the all-cores oracle timing: build the oracle problem of the sample, apply it to its cells
    (private y) and return (apply seconds, y)."""
    import oracle

    (cell_type, coords, cv, p, cn, nnode, kind, ncomp, qdeg, coef, okw, xs, cells) = task
    pb = oracle.Problem(cell_type, coords, cv, p, cn, nnode, kind, ncomp=ncomp, qdeg=qdeg, ucoef=coef, **okw)
    t0 = time.perf_counter()
    y = pb.apply(xs, cells=cells)
    return time.perf_counter() - t0, y


def oracle_rate_all_cores(cases, single, workers):
    """The oracle on all host cores: each operator's sample cells split over `workers` spawned processes, each
    applying the unchanged oracle to its share with a private y, then a reduction.  Wall time = the slowest
    worker's apply plus the reduction; full mesh = the single-core fit's fixed part + the rest scaled by cells."""
    import multiprocessing as mp

    out = []
    with mp.get_context("spawn").Pool(workers) as pool:
        # start every worker before timing; every wait is bounded (a lost worker raises, the pool is terminated)
        pool.map_async(abs, range(workers)).get(timeout=300)
        for c, s in zip(cases, single):
            cv, cn, nodes, nsub = sub_mesh(c, s["sample_cells"])
            verts, cv_local = np.unique(cv, return_inverse=True)
            coef = None if c.get("coef") is None else c["coef"].reshape(-1, c["ncomp"])[nodes].ravel()
            xs = c["x"].reshape(-1, c["ncomp"])[nodes].ravel()
            chunks = np.array_split(np.arange(nsub, dtype=np.int64), workers)
            tasks = [(c["cell_type"], c["mesh"].coords[verts], cv_local.reshape(cv.shape).astype(np.int32), c["p"],
                      cn, nodes.size, FORM_IDS[c["form"]], c["ncomp"], c["qdeg"], coef, c["okw"], xs, ch)
                     for ch in chunks if ch.size]
            res = pool.map_async(_oracle_chunk_apply, tasks).get(timeout=300)
            t0 = time.perf_counter()
            y = np.sum([r[1] for r in res], axis=0)
            wall = max(r[0] for r in res) + (time.perf_counter() - t0)
            ncell = c["mesh"].ncell
            full = s["fixed_s"] + max(wall - s["fixed_s"], 0.0) * ncell / nsub
            out.append(dict(name=c["name"], full_s=full, sample_cells=nsub, wall_s=wall, checksum=float(y.sum())))
    return out


def reference_arm(args, world, rank):
    if rank != 0:
        return
    cases = build_cases(args)
    for _ in range(args.warmup):
        oracle_rate(cases[:1])
    times, samples = [], None
    for _ in range(args.steps):
        r = oracle_rate(cases)
        samples = r
        times.append(sum(o["full_s"] for o in r))
    ndof = sum(c["ndof"] for c in cases)
    step_s = statistics.mean(times)
    value = ndof / step_s / 1e9
    sample_desc = ("per operator the first n/2 and n cells of the mesh (%s); full-mesh time = fixed per-call part + "
                   "per-cell slope x cells" % ", ".join("%s: n=%d" % (o["name"], o["sample_cells"]) for o in samples))
    line = {
        "impl": "reference", "metric": "operator-action GDoF/s", "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "operators": [c["name"] for c in cases]},
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": 1, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def gpu_arm(args, world, rank, local):
    import torch

    from paper_1903_08243_gb300 import build as libbuild

    libbuild.build()
    import paper_1903_08243_gb300 as mfa

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = mfa.Context(local, stream)
    cases = build_cases(args)
    scatter = {"atomic": mfa.MFA_SCATTER_ATOMIC, "colour": mfa.MFA_SCATTER_COLOUR,
               "warp": mfa.MFA_SCATTER_WARP}[args.scatter]
    meshes, spaces, ops = {}, {}, []
    setup_s = {"mesh_upload": 0.0, "space": 0.0, "forms": 0.0}  # wall time, each creation synchronised
    for c in cases:
        mk = (id(c["mesh"]), hashlib.sha1(np.ascontiguousarray(c["cell_vert"])).hexdigest())
        if mk not in meshes:
            t0 = time.perf_counter()
            meshes[mk] = mfa.Mesh(ctx, c["cell_type"], c["mesh"].coords, c["cell_vert"])
            ctx.sync()
            setup_s["mesh_upload"] += time.perf_counter() - t0
        sk = (mk, c["p"], c["ncomp"])
        if sk not in spaces:
            t0 = time.perf_counter()
            spaces[sk] = mfa.Space(meshes[mk], c["p"], c["ncomp"], c["cell_node"], c["nnode"])
            ctx.sync()
            setup_s["space"] += time.perf_counter() - t0
        prec = {"fp64": mfa.MFA_PREC_FP64, "fp32": mfa.MFA_PREC_FP32, "bf16": mfa.MFA_PREC_BF16}[args.precision]
        if c["cell_type"] != 8:
            prec = mfa.MFA_PREC_FP64
        geo = mfa.MFA_GEOM_ONTHEFLY if (args.geometry == "onthefly" and c["cell_type"] == 8) else mfa.MFA_GEOM_STORED
        t0 = time.perf_counter()
        rule = mfa.MFA_RULE_SYMMETRIC if (args.rule == "symmetric" and c["cell_type"] in (3, 4)) else mfa.MFA_RULE_AUTO
        form = mfa.Form(spaces[sk], FORM_IDS[c["form"]], scatter=scatter, qdeg=c["qdeg"] if c["cell_type"] == 8 else 0,
                        precision=prec, geometry=geo, rule=rule, **c["kw"])
        ctx.sync()
        form_s = time.perf_counter() - t0
        setup_s["forms"] += form_s
        x = torch.from_numpy(c["x"]).to("cuda")
        y = torch.empty_like(x)
        if c.get("coef") is not None:
            form.set_coefficient(torch.from_numpy(c["coef"]).to("cuda"))
        ops.append(dict(case=c, form=form, x=x, y=y, info=form.info(), setup_ms=form_s * 1e3))
    ctx.sync()
    # autotuner: every compiled launch configuration of each form is timed, the fastest kept
    tune_s = 0.0
    if not args.no_autotune:
        t0 = time.perf_counter()
        for o in ops:
            default_cfg = o["form"].config()
            tried = o["form"].autotune(o["x"], o["y"], reps=3)
            default_ms = next(c.ms for c in tried if (c.variant, c.cells_per_block, c.scatter) ==
                              (default_cfg.variant, default_cfg.cells_per_block, default_cfg.scatter))
            o["tune"] = dict(o["form"].config().as_dict(), default_ms=default_ms, configs_tried=len(tried))
            o["info"] = o["form"].info()
        tune_s = time.perf_counter() - t0
    for o in ops:
        o["cfg"] = o["form"].config()
    ctx.sync()
    probe_tflops, probe_mhz = mfa.mfa_probe_fp64_fma(ctx.h)  # the measured FP64 FMA rate (outside the timing)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    launches_per_step = sum(o["info"].ncolours if o["info"].scatter == mfa.MFA_SCATTER_COLOUR else 1 for o in ops)

    def step(events=None, s=None):
        s = s or stream
        for i, o in enumerate(ops):
            if events is not None:
                events[i][0].record(s)
            mfa.mfa_apply(ctx.h, o["form"].h, o["x"], o["y"], False)
            if events is not None:
                events[i][1].record(s)

    graphs = None
    if args.graph:
        # one graph per operator so that events can bracket each replay
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        mfa.mfa_set_stream(ctx.h, side)
        with torch.cuda.stream(side):
            step(s=side)
        side.synchronize()
        graphs = []
        for o in ops:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                mfa.mfa_apply(ctx.h, o["form"].h, o["x"], o["y"], False)
            graphs.append(g)
        mfa.mfa_set_stream(ctx.h, stream)
        torch.cuda.synchronize()

    def run_step(events=None):
        if graphs is None:
            step(events)
            return
        for i, g in enumerate(graphs):
            if events is not None:
                events[i][0].record(stream)
            g.replay()
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        run_step()
    ctx.sync()
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in ops]
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 flush between steps, outside the per-operator events
        run_step(ev[k])
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    time.sleep(0.3)
    clocks = sampler.stop()
    ctx.sync()
    per_op_ms = [statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
                 for i in range(len(ops))]
    step_ms = allreduce_max(world, sum(per_op_ms))
    ndof_step = sum(o["case"]["ndof"] for o in ops)
    value = world * ndof_step / (step_ms / 1e3) / 1e9

    # dominant kernel roofline (FP64 pipe)
    i_dom = int(np.argmax(per_op_ms))
    dom = ops[i_dom]
    achieved = dom["info"].flops / (per_op_ms[i_dom] / 1e3) / 1e12
    if dom["case"]["cell_type"] == 8:
        ksrc, kbase = (("hex_vector.cuh", "hexv::apply_kernel") if dom["case"]["ncomp"] == 3
                       else VARIANT_KERNELS[dom["cfg"].variant])
        kh = kernel_hash(ksrc)
        kname = kbase + "<n=%d,%s,cb=%d>" % (dom["case"]["p"] + 1, dom["case"]["form"], dom["cfg"].cells_per_block)
    else:
        moment = dom["case"]["p"] == 2 and dom["case"]["form"] in ("hyper_res", "hyper_jac")
        kname = "simplex_dense_kernel<DIM=3, %s>" if dom["case"]["p"] >= 3 else (
            "tet_moment_kernel<%s>" if moment else "tet_apply_kernel<%s>")
        if dom["case"]["cell_type"] == 40:
            kname = "quad_apply_kernel<%s>"
        elif dom["case"]["cell_type"] == 3:
            kname = ("tri_cell_kernel<%s>" if dom["cfg"].variant == 5 else "simplex_dense_kernel<DIM=2, %s>")
        kh, kname = None, kname % dom["case"]["name"]
    traffic = NCU_TRAFFIC.get((kh, dom["case"]["name"]))
    if args.workload == "hex" and args.precision != "fp64":
        # FP32/BF16 contractions: bound by HBM bandwidth (algorithmic bytes of the dominant operator)
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        gbs = dom["info"].bytes / (per_op_ms[i_dom] / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                    "traffic": traffic, "operator": dom["case"]["name"], "kernel": kname,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                    "algorithmic_bytes_per_launch": dom["info"].bytes, "kernel_sha1": kh}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic, "operator": dom["case"]["name"],
                    "kernel": kname,
                    "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (FP64 pipe; recipe unit counts)",
                    "algorithmic_flops_per_launch": dom["info"].flops,
                    "executed_flops_per_launch": dom["info"].flops_executed,
                    "frac_executed": dom["info"].flops_executed / (per_op_ms[i_dom] / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                    "algorithmic_bytes_per_launch": dom["info"].bytes, "kernel_sha1": kh,
                    "fp64_probe": {"tflops": probe_tflops, "sm_mhz": probe_mhz,
                                   "frac_of_derived_peak": probe_tflops / FP64_PEAK_TFLOPS,
                                   "source": "mfa_probe_fp64_fma: 8 independent FMA chains per thread, one wave "
                                             "of blocks per SM, CUDA events"}}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if args.e2e_steps > 0:
        hx = [torch.from_numpy(o["case"]["x"]).pin_memory() for o in ops]
        hy = [torch.empty_like(h).pin_memory() for h in hx]
        forms_h = [o["form"].h for o in ops]
        for _ in range(max(1, args.warmup)):  # warm-up calls, untimed like the device leg's: staging buffers,
            mfa.mfa_apply_host_many(ctx.h, forms_h, hx, hy)  # copy streams, first touch of the pinned pages
        # per step also the span on the context stream between events recorded before and after the call (the
        # call returns once its copies are done): a step whose wall time exceeds its span lost time on the host
        spans = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.e2e_steps)]
        barrier(world)
        t0 = time.perf_counter()
        marks = []
        for k in range(args.e2e_steps):
            spans[k][0].record(stream)
            mfa.mfa_apply_host_many(ctx.h, forms_h, hx, hy)
            spans[k][1].record(stream)
            marks.append(time.perf_counter())
        dt = (time.perf_counter() - t0) / args.e2e_steps
        dt = allreduce_max(world, dt)
        torch.cuda.synchronize()
        each = [1e3 * (b - a) for a, b in zip([t0] + marks[:-1], marks)]
        span_each = [a.elapsed_time(b) for a, b in spans]
        e2e = {"value": world * ndof_step / dt / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * ndof_step,
               "d2h_bytes_per_step": 8 * ndof_step, "ms_per_step": dt * 1e3, "ms_each_step": each,
               "stream_span_ms_each_step": span_each,
               "path": "mfa_apply_host_many: pinned host buffers, copies overlapped with the applies",
               "host_link": host_link_gbs()}

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_rate(cases, samples=SAMPLE_CPU_LEG)
        full_s = sum(o["full_s"] for o in r)
        cpu = {"value": ndof_step / full_s / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
               "sample": "per operator the first n/2 and n cells of the mesh (%s), each timed once; full-mesh time = "
                         "fixed per-call part + per-cell slope x cells" % ", ".join(
                             "%s n=%d %.2fs" % (o["name"], o["sample_cells"], o["sample_s"]) for o in r)}
        # the same oracle on every host core: cells split over spawned worker processes (private y, reduction)
        try:
            avail = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
            workers = max(1, min(avail, 64))  # the cores this process may run on
            ra = oracle_rate_all_cores(cases, r, workers)
            full_a = sum(o["full_s"] for o in ra)
            cpu_all = {"value": ndof_step / full_a / 1e9, "unit": "GDoF/s", "cores": workers, "kind": "oracle",
                       "sample": "the single-core samples split over %d spawned processes (each the unchanged "
                                 "oracle on its share of the cells, private y, then a reduction); full-mesh time = "
                                 "the single-core fixed part + the rest scaled by cells" % workers}
        except Exception as e:  # the all-cores figure is context; its failure must not cost the line
            cpu_all = {"value": None, "error": "%s: %s" % (type(e).__name__, e)}

    per_op = []
    for o, ms in zip(ops, per_op_ms):
        per_op.append({"operator": o["case"]["name"], "ndof": o["case"]["ndof"], "ms": ms,
                       "gdof_s": o["case"]["ndof"] / ms / 1e6, "gflop_s": o["info"].flops / ms / 1e6,
                       "frac_fp64": o["info"].flops / ms / 1e9 / FP64_PEAK_TFLOPS,
                       "frac_fp64_executed": o["info"].flops_executed / ms / 1e9 / FP64_PEAK_TFLOPS,
                       "ncolours": o["info"].ncolours,
                       "launch": dict(o["cfg"].as_dict(), ms=None), "tune": o.get("tune"),
                       "setup_ms": o["setup_ms"]})
    if rank == 0:
        cfg = {"workload": workload_name(args), "operators": [c["name"] for c in cases], "scatter": args.scatter,
               "ndof_per_step": ndof_step, "graph_replay": bool(args.graph),
               "l2": "flushed between steps (256 MiB write outside the timed events)",
               "parallelism": "replicas" if world > 1 else "single",
               "setup_ms": {k: v * 1e3 for k, v in setup_s.items()},
               "setup_note": "outside the timed region: mesh upload; space (map upload, colouring); forms (tables, "
                             "stored geometric factors); each synchronised, wall clock",
               "autotune": None if args.no_autotune else "every compiled launch configuration timed (3 reps, "
                                                          "warm L2) before warm-up; %.2f s" % tune_s}
        if args.workload == "hex":
            cfg.update({"mesh": "%d^3 hex, interior vertices perturbed U[-0.1h,0.1h], seed 1" % args.nx,
                        "quadrature": "p+1 Gauss points per direction", "geometry": "stored FP64 G per point",
                        "input": "x ~ U[-1,1) seed 1"})
        elif args.workload == "hex-vector":
            cfg.update({"mesh": "%d^3 hex, interior vertices perturbed U[-0.1h,0.1h], seed 1" % args.nx,
                        "quadrature": "p+1 Gauss points per direction",
                        "geometry": "stored FP64 J^-1 and w|det J| per point", "lambda": 1.0, "mu": 1.0,
                        "input": "residual and coefficient: sinusoid displacement (8 terms, amplitude 0.05, seed 2) "
                                 "on the node grid; elasticity and Jacobian: x ~ U[-1,1) seed 1"})
        elif args.workload == "planar":
            cfg.update({"mesh": "%d^2 quads and %d^2 boxes x 2 triangles, unit square, interior vertices perturbed "
                                "U[-0.1h,0.1h], seed 1" % (args.nx, args.nx // 2),
                        "quadrature": "quads: p+1 Gauss points per direction; triangles: the cheapest rule exact for "
                                      "the polynomial integrand (Table 2's symmetric rules up to degree 6)",
                        "vector forms": "plane strain, lambda = mu = 1",
                        "input": "scalar x ~ U[-1,1) seed 0; vector: sinusoid displacement seed 2"})
        elif args.workload == "tet-pk":
            cfg.update({"mesh": "%d^3 boxes x 6 Kuhn tets" % args.nx,
                        "quadrature": "the cheapest rule exact for the polynomial integrand (degree 2p mass/Helmholtz, "
                                      "2p-2 Laplace/elasticity): Table 2's symmetric rules up to degree 6 (P3: 24 / "
                                      "14 points), collapsed Gauss-Jacobi above",
                        "basis": "equispaced lattice Lagrange", "lambda": 1.0, "mu": 1.0,
                        "input": "scalar x ~ U[-1,1) seed 0; vector: sinusoid displacement seed 2"})
        elif args.workload == "tet-p1-mass":
            cfg.update({"mesh": "%d^3 boxes x 6 Kuhn tets" % args.nx, "quadrature": "degree 2",
                        "input": "x ~ U[-1,1) seed 0"})
        else:
            cfg.update({"mesh": "%d^3 boxes x 6 Kuhn tets" % args.nx,
                        "quadrature": "elasticity: the 4-point degree-2 rule (exact); neo-Hookean: degree 4, the "
                                      "27-point collapsed rule, or Table 2's 14-point symmetric rule with --rule "
                                      "symmetric",
                        "lambda": 1.0, "mu": 1.0, "input": "sinusoid displacement, 8 terms, amplitude 0.05, seed 2"})
        line = {
            "metric": "operator-action GDoF/s", "value": value, "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "data": "synthetic", "config": cfg,
            "dtype": {"fp64": "f64", "fp32": "f32 (FP64 vectors)", "bf16": "bf16 operands, f32 accumulation"}[
                args.precision if args.workload == "hex" else "fp64"],
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps, "wall_s_timed_region": t_wall,
            "ms_per_step_bracketed": t_wall / args.steps * 1e3,
            "timing": "ms_per_step = sum over operators of the median (over steps) of each operator's CUDA-event "
                      "time; ms_per_step_bracketed = wall time of the timed steps / steps (includes the L2 flush)",
            "per_operator": per_op,
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ sharded hex workload (N > 1)

def sharded_operators(world, rank, nx, degrees, forms, make_part, to_tensor):
    """This rank's operators of the z-slab sharded hex workload (weak scaling): the box [0,1]^2 x [0, N] of
    nx * nx * (N nx) perturbed hexahedra, rank r holding cell layers [r nx, (r + 1) nx), so that every rank has
    the single-GPU workload's nx^3 cells.  For each degree and form: the slab's halo plan, its two parts (the
    cells touching a node shared with a neighbour, and the rest) built by make_part(mesh, plan, cells, p, form),
    the rank's slice of the global seeded x, and y.  Part objects have apply(x, y, accumulate)."""
    from paper_1903_08243_gb300 import dist as mdist

    mesh = fi.hex_slab_mesh(nx, nx * world, rank * nx, nx, perturb=0.1, seed=1)
    out = []
    for p in degrees:
        plan = mdist.slab_plan(nx, nx, p, world, rank)
        x = to_tensor(fi.uniform_vector(plan.l2g.size, seed=1, start=int(plan.l2g[0])))
        for f in forms:
            parts = {name: (make_part(mesh, plan, cells, p, f) if cells.size else None)
                     for name, cells in (("boundary", plan.boundary_cells), ("interior", plan.interior_cells))}
            out.append(dict(name="Q%d %s" % (p, f), p=p, form=f, plan=plan, parts=parts, x=x, y=x.clone(),
                            ndof_owned=int(plan.owned.sum())))
    return out


def sharded_step(op, plan, halo_ops, on_interior=None):
    """One distributed action y = A x of a sharded operator on this rank: import x at the ghost plane, apply the
    boundary cells, post the reverse exchange of their partial sums, apply the interior cells while it is in
    flight, then add the received partial sums into the owned plane (on_interior(apply) wraps the interior
    apply, e.g. to time it)."""
    from paper_1903_08243_gb300 import dist as mdist

    b, i = op["parts"]["boundary"], op["parts"]["interior"]

    def apply_boundary(x, y):
        if b is None:
            y.zero_()
        else:
            b.apply(x, y, False)
        return y

    def apply_interior(x, y):
        if i is not None:
            (on_interior or (lambda fn: fn()))(lambda: i.apply(x, y, True))

    return mdist.distributed_apply_overlapped(plan, apply_boundary, apply_interior, op["x"], halo_ops, y=op["y"],
                                              refresh=False)


def sharded_hex_arm(args, world, rank, local):
    """The hex workload sharded over N GPUs (z-slabs, halo exchange by NCCL point-to-point messages, the reverse
    exchange overlapping the interior cells); weak scaling, nx^3 cells per GPU."""
    import torch

    from paper_1903_08243_gb300 import build as libbuild
    from paper_1903_08243_gb300 import dist as mdist

    libbuild.build()
    import paper_1903_08243_gb300 as mfa

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = mfa.Context(local, stream)
    halo = mdist.LibraryHaloOps(ctx)
    args.nx = args.nx or 64
    degrees = [int(p) for p in args.degrees.split(",")]
    forms = args.forms.split(",")
    keep = []

    class Part:
        def __init__(self, mesh, plan, cells, p, f):
            m = mfa.Mesh(ctx, mfa.MFA_CELL_HEX8, mesh.coords, np.ascontiguousarray(mesh.cell_vert[cells]))
            sp = mfa.Space(m, p, 1, np.ascontiguousarray(plan.local_cell_node[cells]), plan.l2g.size)
            self.form = mfa.Form(sp, FORM_IDS[f], k2=1.0)
            keep.append((m, sp))

        def apply(self, x, y, accumulate):
            mfa.mfa_apply(ctx.h, self.form.h, x, y, accumulate)

    t0 = time.perf_counter()
    ops = sharded_operators(world, rank, args.nx, degrees, forms, Part, lambda a: torch.from_numpy(a).cuda())
    plans = {}
    for o in ops:
        if o["p"] not in plans:
            plans[o["p"]] = mdist.device_plan(o["plan"], "cuda")
        o["dplan"] = plans[o["p"]]
    ctx.sync()
    setup_s = time.perf_counter() - t0
    if not args.no_autotune:
        for o in ops:
            for part in o["parts"].values():
                if part is not None:
                    part.form.autotune(o["x"], o["y"], reps=3)
    ctx.sync()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    kev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in ops]
           for _ in range(args.steps)]
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in ops]
          for _ in range(args.steps)]

    def run_step(k=None):
        for i, o in enumerate(ops):
            if k is not None:
                ev[k][i][0].record(stream)

            def timed(fn, k=k, i=i):
                if k is not None:
                    kev[k][i][0].record(stream)
                fn()
                if k is not None:
                    kev[k][i][1].record(stream)
            sharded_step(o, o["dplan"], halo, timed)
            if k is not None:
                ev[k][i][1].record(stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        run_step()
    ctx.sync()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        run_step(k)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    time.sleep(0.3)
    clocks = sampler.stop()
    ctx.sync()
    per_op_ms = [statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
                 for i in range(len(ops))]
    kern_ms = [statistics.median(kev[k][i][0].elapsed_time(kev[k][i][1]) for k in range(args.steps))
               if ops[i]["parts"]["interior"] is not None else 0.0 for i in range(len(ops))]
    step_ms = allreduce_max(world, sum(per_op_ms))
    ndof_rank = sum(o["ndof_owned"] for o in ops)
    ndof_step = ndof_rank
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([ndof_rank], dtype=torch.int64, device="cuda")
        dist.all_reduce(t)
        ndof_step = int(t.item())
    value = ndof_step / (step_ms / 1e3) / 1e9
    i_dom = int(np.argmax(kern_ms))
    dom = ops[i_dom]["parts"]["interior"]
    info = dom.form.info() if dom is not None else None
    roofline = None
    if info is not None and kern_ms[i_dom] > 0:
        achieved = info.flops / (kern_ms[i_dom] / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "operator": ops[i_dom]["name"],
                    "scope": "the interior cells' apply kernel of rank %d (CUDA events on the context stream)" % rank,
                    "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (FP64 pipe; recipe unit counts)",
                    "frac_executed": info.flops_executed / (kern_ms[i_dom] / 1e3) / 1e12 / FP64_PEAK_TFLOPS}

    # end to end: each step copies the rank's x in from pinned host memory and its y back
    e2e = None
    if args.e2e_steps > 0:
        hx = [torch.from_numpy(o["x"].cpu().numpy()).pin_memory() for o in ops]
        hy = [torch.empty_like(h).pin_memory() for h in hx]

        def e2e_step():
            for o, xh, yh in zip(ops, hx, hy):
                o["x"].copy_(xh, non_blocking=True)
                sharded_step(o, o["dplan"], halo)
                yh.copy_(o["y"], non_blocking=True)
            torch.cuda.synchronize()

        for _ in range(max(1, args.warmup)):  # untimed, like the device leg's warm-up
            e2e_step()
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        dt = allreduce_max(world, (time.perf_counter() - t0) / args.e2e_steps)
        nbytes = 8 * sum(o["x"].numel() for o in ops)
        e2e = {"value": ndof_step / dt / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "ms_per_step": dt * 1e3,
               "path": "per rank and operator: pinned x copied in, the sharded action (halo exchange included), y "
                       "copied out"}
    # this rank's library launches per step: halo pack/unpack per peer and direction, and the two parts' applies
    launches = sum(len(o["plan"].send_import) + len(o["plan"].recv_import) + len(o["plan"].send_reverse) +
                   len(o["plan"].recv_reverse) + sum(part is not None for part in o["parts"].values()) for o in ops)
    if rank == 0:
        halo_nodes = {o["name"]: int(sum(ids.size for ids in o["plan"].recv_import.values())) for o in ops}
        line = {
            "metric": "operator-action GDoF/s", "value": value, "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args) + "-sharded", "operators": [o["name"] for o in ops],
                       "parallelism": "sharded", "ndof_per_step": ndof_step,
                       "mesh": "[0,1]^2 x [0,%d] as %d x %d x %d hexahedra (h = 1/%d), interior vertices perturbed "
                               "U[-0.1h,0.1h], seed 1; rank r holds cell layers [%d r, %d (r+1))"
                               % (world, args.nx, args.nx, args.nx * world, args.nx, args.nx, args.nx),
                       "exchange": "NCCL point-to-point, one grouped exchange per direction: x imported at the "
                                   "ghost node plane before the apply; the boundary cells' partial sums sent back "
                                   "while the interior cells are applied",
                       "halo_nodes_rank0": halo_nodes,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "setup_s": setup_s, "input": "the rank's slice of the global x ~ U[-1,1) seed 1"},
            "roofline": roofline, "cpu_baseline": None, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches * args.steps, "wall_s_timed_region": t_wall,
            "per_operator": [{"operator": o["name"], "ms": ms, "interior_kernel_ms": km}
                             for o, ms, km in zip(ops, per_op_ms, kern_ms)],
        }
        print(json.dumps(line), flush=True)


def batched_specs(nops, seed=3):
    """Operator list of the batched workload: degree ~ U{1..8}, cells per side ~ U{8..48}."""
    deg = fi.randint(seed, 0xDE6, nops, 1, 8)
    side = fi.randint(seed, 0x51DE, nops, 8, 48)
    return [(int(p), int(n)) for p, n in zip(deg, side)]


BATCHED_SAMPLE_DOFS = {1: 64, 2: 64, 3: 48, 4: 32, 5: 24, 6: 16, 7: 12, 8: 8}


def batched_oracle_leg(hosts, y_host, world):
    """Per operator: the FP64 oracle on the cells touching a few random dofs (seeded), its time (CPU baseline,
    one core, scaled by cells to the whole operator) and the relative L2 and max errors of the GPU result at those
    dofs (the reference there is complete: every cell that adds into them is applied)."""
    import oracle

    errs, full_s, ncells, nsample = [], 0.0, 0, 0
    for i, h in enumerate(hosts):
        rng = np.random.default_rng(4000 + i)
        dofs = rng.choice(h["nnode"], size=min(BATCHED_SAMPLE_DOFS[h["p"]], h["nnode"]), replace=False)
        cells = np.nonzero(np.isin(h["cell_node"], dofs).any(axis=1))[0]
        pb = oracle.Problem(oracle.HEX, h["mesh"].coords, h["mesh"].cell_vert, h["p"], h["cell_node"], h["nnode"],
                            oracle.HELMHOLTZ, k2=1.0)
        t0 = time.perf_counter()
        ref = pb.apply(h["x"], cells=cells)
        dt = time.perf_counter() - t0
        full_s += dt * h["mesh"].ncell / cells.size
        ncells += cells.size
        nsample += dofs.size
        y, r = y_host[i][dofs], ref[dofs]
        errs.append({"rel_l2": float(np.linalg.norm(y - r) / np.linalg.norm(r)),
                     "max_rel": float(np.abs(y - r).max() / np.abs(r).max())})
    ndof = sum(h["nnode"] for h in hosts)
    cpu = {"value": world * ndof / full_s / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
           "sample": "per operator the cells touching %d random dofs (8 to 64 by degree; %d cells in all), timed "
                     "once and scaled by cells to the whole operator" % (nsample, ncells)}
    acc = {"reference": "FP64 oracle (oracle/) on the cells touching the sampled dofs", "dofs_sampled": nsample,
           "per_operator": errs, "max_rel_l2": max(e["rel_l2"] for e in errs),
           "max_max_rel": max(e["max_rel"] for e in errs)}
    return cpu, acc


def batched_arm(args, world, rank, local):
    import torch

    from paper_1903_08243_gb300 import build as libbuild

    libbuild.build()
    import paper_1903_08243_gb300 as mfa

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = mfa.Context(local, stream)
    prec = {"fp64": mfa.MFA_PREC_FP64, "fp32": mfa.MFA_PREC_FP32, "bf16": mfa.MFA_PREC_BF16}[args.precision]
    specs = batched_specs(args.nops)
    keep, forms, xs, ys, infos, hosts = [], [], [], [], [], []
    for i, (p, n) in enumerate(specs):
        mesh = fi.hex_box_mesh(n, perturb=0.1, seed=1000 + i)
        cell_node, nnode = fi.hex_node_map(n, p)
        m = mfa.Mesh(ctx, mfa.MFA_CELL_HEX8, mesh.coords, mesh.cell_vert)
        sp = mfa.Space(m, p, 1, cell_node, nnode)
        f = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, k2=1.0, precision=prec)
        xh = fi.uniform_vector(nnode, seed=2000 + i)
        x = torch.from_numpy(xh).cuda()
        keep.append((m, sp))
        forms.append(f)
        xs.append(x)
        ys.append(torch.empty_like(x))
        infos.append(f.info())
        hosts.append(dict(p=p, n=n, mesh=mesh, cell_node=cell_node, nnode=nnode, x=xh))
    ctx.sync()
    batch = mfa.mfa_batch_create(ctx.h, [f.h for f in forms], xs, ys)
    ngroups, nsingles = mfa.mfa_batch_info(batch)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.fill_(1.0)
        mfa.mfa_batch_apply(ctx.h, batch)
    ctx.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        mfa.mfa_batch_apply(ctx.h, batch)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    time.sleep(0.3)
    clocks = sampler.stop()
    ctx.sync()
    step_ms = allreduce_max(world, statistics.median(a.elapsed_time(b) for a, b in ev))
    ndof = sum(i.ndof for i in infos)
    value = world * ndof / (step_ms / 1e3) / 1e9
    y_host = [y.cpu().numpy() for y in ys]

    # end to end through the C ABI with host buffers: every operator's x copied in and y copied out each step
    e2e = None
    if args.e2e_steps > 0:
        hx = [torch.from_numpy(h["x"]).pin_memory() for h in hosts]
        hy = [torch.empty_like(t).pin_memory() for t in hx]
        forms_h = [f.h for f in forms]
        for _ in range(max(1, args.warmup)):  # warm-up calls, untimed like the device leg's: staging buffers,
            mfa.mfa_apply_host_many(ctx.h, forms_h, hx, hy)  # copy streams, first touch of the pinned pages
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            mfa.mfa_apply_host_many(ctx.h, forms_h, hx, hy)
        dt = allreduce_max(world, (time.perf_counter() - t0) / args.e2e_steps)
        e2e = {"value": world * ndof / dt / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * ndof,
               "d2h_bytes_per_step": 8 * ndof, "ms_per_step": dt * 1e3,
               "path": "mfa_apply_host_many: pinned FP64 host buffers, copies overlapped with the applies (one "
                       "launch per operator, not the grouped graph)", "host_link": host_link_gbs()}

    # CPU baseline and accuracy: the FP64 oracle on the cells touching a few random dofs of every operator, timed
    # (one core), and the GPU result at those dofs compared with it
    cpu, accuracy = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, accuracy = batched_oracle_leg(hosts, y_host, world)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    total_bytes = sum(i.bytes for i in infos)
    total_flops = sum(i.flops for i in infos)
    if prec == mfa.MFA_PREC_FP64:
        achieved = total_flops / (step_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None}
    else:
        achieved = total_bytes / (step_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": None,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}
    roofline.update({"scope": "whole batch graph (all grouped launches) per replay",
                     "algorithmic_bytes_per_step": total_bytes, "algorithmic_flops_per_step": total_flops})
    if rank == 0:
        line = {
            "metric": "operator-action GDoF/s", "value": value, "unit": "GDoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16 operands, f32 accumulate"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "batched-%d-hex-helmholtz-%s" % (args.nops, args.precision),
                       "operators": "%d Helmholtz (k2=1) operators, degree ~ U{1..8}, n^3 perturbed hexes with n ~ U{8..48}, seed 3" % args.nops,
                       "degrees": [p for p, _ in specs], "sides": [n for _, n in specs], "ndof_per_step": ndof,
                       "launch": "one CUDA graph replay: %d grouped persistent launches + %d single launches" % (ngroups, nsingles),
                       "l2": "flushed between steps (256 MiB write outside the timed events)"},
            "roofline": roofline, "clocks": clocks, "gpu_launches": (ngroups + nsingles) * args.steps,
            "error_vs_oracle": accuracy, "wall_s_timed_region": t_wall,
            "ms_per_step_bracketed": t_wall / args.steps * 1e3, "cpu_baseline": cpu, "e2e": e2e,
        }
        print(json.dumps(line), flush=True)
    mfa.mfa_batch_destroy(batch)


def pcg_arm(args, world, rank, local):
    """Time to ||b - A x|| <= 1e-8 ||b||: FP64 Jacobi-PCG, mixed FCG (FP32 Jacobi inner loop), and mixed
    FCG with the learned linear preconditioner in the inner loop (training time reported separately)."""
    import torch

    from paper_1903_08243_gb300 import build as libbuild

    libbuild.build()
    import paper_1903_08243_gb300 as mfa

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = mfa.Context(local, stream)
    nx, p = (args.nx or 64), 4
    mesh = fi.hex_box_mesh(nx, perturb=0.1, seed=1)
    cell_node, nnode = fi.hex_node_map(nx, p)
    m = mfa.Mesh(ctx, mfa.MFA_CELL_HEX8, mesh.coords, mesh.cell_vert)
    sp = mfa.Space(m, p, 1, cell_node, nnode)
    A64 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, k2=1.0)
    iprec = {"fp64": mfa.MFA_PREC_FP64, "fp32": mfa.MFA_PREC_FP32, "bf16": mfa.MFA_PREC_BF16}[args.inner_precision]
    A32 = mfa.Form(sp, mfa.MFA_FORM_HELMHOLTZ, k2=1.0, precision=iprec)
    M64 = mfa.Form(sp, mfa.MFA_FORM_MASS)
    rtol = 1e-8
    # the solver's operators take the autotuner's launch configuration (setup, outside every timed solve)
    tune_x = torch.rand(sp.ndof, dtype=torch.float64, device="cuda")
    tune_y = torch.empty_like(tune_x)
    tuned = {}
    for name, F in (("fp64 outer", A64), ("inner", A32)):
        if not args.no_autotune:
            F.autotune(tune_x, tune_y)
        tuned[name] = F.config().as_dict()
    del tune_x, tune_y

    def grf_rhs(seed):
        f = torch.from_numpy(fi.grf_lattice(nx * p + 1, seed=seed)).cuda()
        b = M64.apply(f)  # b = M f_h
        ctx.sync()
        return b

    # ---- training data: (r, e) pairs from plain CG iterates.  "grf": right-hand sides like the test
    # ones, reference solution by the mixed solver; "white": manufactured solutions x* ~ U[-1,1) per dof,
    # b = A x*, whose early plain-CG errors span the whole spectrum (the part a local preconditioner can act on);
    # "mixed": both, so that the loss also sees the smooth late errors that set the smallest eigenvalue of M A.
    t0 = time.perf_counter()
    rs, es = [], []
    kinds = {"grf": ["grf"], "white": ["white"], "mixed": ["white", "grf"]}[args.train_data]
    its_of = {"grf": (2, 6, 20, 60, 150), "white": (0, 1, 2, 4, 8, 16)}
    its = tuple(k for kind in kinds for k in its_of[kind])
    for kind in kinds:
        for j in range(args.train_rhs):
            if kind == "grf":
                b = grf_rhs(300 + j)
                xs = torch.zeros_like(b)
                mfa.mfa_fcg_mixed(ctx.h, A64.h, A32.h, args.inner, b, xs, 1e-10, 5000)
            else:
                xs = torch.from_numpy(fi.uniform_vector(nnode, seed=300 + j)).cuda()
                b = A64.apply(xs)
            for k in its_of[kind]:
                x = torch.zeros_like(b)
                mfa.mfa_cg(ctx.h, A32.h, mfa.MFA_PC_NONE, b, x, 1e-30, k)  # k plain CG steps
                r = b - A64.apply(x)
                rs.append(r.float())
                es.append((xs - x).float())
    ctx.sync()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    pc = mfa.mfa_precond_create(ctx.h, A64.h, 5, mode=mfa.MFA_PRECOND_LINEAR)
    loss_first, loss_last = mfa.mfa_precond_train(ctx.h, pc, A32.h, rs, es, args.train_steps, args.train_lr)
    ctx.sync()
    t_train = time.perf_counter() - t0
    del rs, es

    # spectrum of the preconditioned operator (untimed): Ritz values of M A from the Lanczos coefficients of
    # PCG, with M = Jacobi and M = the learned linear preconditioner (symmetric positive definite)
    dA = A64.diagonal()
    ctx.sync()

    def apply_jacobi(r):
        return r / dA

    def apply_learned(r):
        z = torch.empty_like(r, dtype=torch.float32)
        mfa.mfa_precond_apply(ctx.h, pc, r.float(), z)
        return z.double()

    b_spec = grf_rhs(399)
    spectrum = {"iterations": args.lanczos}
    for name, apply_m in (("jacobi", apply_jacobi), ("learned", apply_learned)):
        lo, hi = pcg_ritz_extremes(lambda v: A64.apply(v), apply_m, b_spec, args.lanczos)
        spectrum[name] = {"lambda_min": lo, "lambda_max": hi, "kappa": hi / lo}

    rows = []
    sampler = ClockSampler(local)
    sampler.start()
    methods = ("jacobi_pcg_fp64", "fcg_mixed", "fcg_learned", "fcg_learned_fallback")
    for r in range(args.nrhs + 1):  # the first solve of each method warms up and is not reported
        b = grf_rhs(400 + r)
        res = {}
        for name in methods:
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fb = 0
            if name == "jacobi_pcg_fp64":
                rc, it, rel = mfa.mfa_cg(ctx.h, A64.h, mfa.MFA_PC_JACOBI, b, x, rtol, 20000)
                inner = 0
            elif name == "fcg_mixed":
                rc, it, inner, rel = mfa.mfa_fcg_mixed(ctx.h, A64.h, A32.h, args.inner, b, x, rtol, 5000)
            else:  # the learned solver on its own, then with the in-solve fallback to the Jacobi inner loop
                rc, it, inner, rel, fb = mfa.mfa_fcg_learned(ctx.h, A64.h, A32.h, pc, args.inner, b, x, rtol, 5000,
                                                             fallback=name.endswith("fallback"),
                                                             raise_on_breakdown=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            true_rel = float(torch.linalg.norm(b - A64.apply(x)) / torch.linalg.norm(b))
            res[name] = {"seconds": dt, "iterations": it, "inner_iterations": inner, "relres": rel,
                         "true_relres": true_rel, "status": rc, "converged": bool(true_rel <= 1.01 * rtol),
                         "fallback": fb}
        if r > 0:
            rows.append(res)
    clocks = sampler.stop()
    mfa.mfa_precond_destroy(pc)
    tj = statistics.mean(r["jacobi_pcg_fp64"]["seconds"] for r in rows)
    tm = statistics.mean(r["fcg_mixed"]["seconds"] for r in rows)
    tl = statistics.mean(r["fcg_learned"]["seconds"] for r in rows)
    tlf = statistics.mean(r["fcg_learned_fallback"]["seconds"] for r in rows)
    learned_converged = all(r["fcg_learned"]["converged"] for r in rows)
    if rank == 0:
        line = {
            "metric": "PCG time-to-1e-8", "value": tl, "unit": "s", "n_gpus": world, "steps": args.nrhs,
            "warmup": 1, "ms_per_step": tl * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 outer / %s inner" % args.inner_precision, "data": "synthetic",
            "config": {"workload": "pcg-hex%d^3-Q4-helmholtz-grf" % nx, "ndof": nnode,
                       "rhs": "b = M f_h, f a Gaussian random field (256 random Fourier features, correlation length 0.1) "
                              "on the node lattice; training seeds 300.., test seeds 401..",
                       "stop": "FP64 ||b - A x||_2 <= 1e-8 ||b||_2 from x = 0",
                       "operators": tuned,
                       "learned": "flexible CG (FP64 operator) preconditioned by %d steps of PCG with the %s operator "
                                  "and the learned linear element preconditioner" % (args.inner, args.inner_precision),
                       "training": {"data": args.train_data, "rhs": args.train_rhs, "plain_cg_iterates": list(its),
                                    "steps": args.train_steps,
                                    "lr": args.train_lr, "data_seconds": t_data, "train_seconds": t_train,
                                    "loss_first (Jacobi step)": loss_first, "loss_last": loss_last}},
            "value_is": "the learned solver on its own (no fallback to the Jacobi inner loop)%s" % (
                "" if learned_converged else "; it did NOT reach 1e-8 on every right-hand side within 5000 outer "
                                             "iterations, so the value is a time to the iteration limit"),
            "jacobi_pcg_fp64_seconds": tj, "fcg_mixed_jacobi_seconds": tm, "fcg_learned_seconds": tl,
            "fcg_learned_with_fallback_seconds": tlf,
            "fallback_used": [r["fcg_learned_fallback"]["fallback"] for r in rows],
            "speedup_vs_jacobi_pcg_fp64": tj / tl, "learned_gain_vs_jacobi_inner": tm / tl,
            "learned_beats_jacobi_inner": bool(learned_converged and tl < tm),
            "spectrum_of_MA": spectrum, "solves": rows,
            "clocks": clocks, "roofline": None, "cpu_baseline": None, "e2e": None,
        }
        print(json.dumps(line), flush=True)


def pcg_ritz_extremes(apply_a, apply_m, b, iters):
    """Smallest and largest Ritz values of M A after `iters` PCG steps from x = 0 (the Lanczos tridiagonal of the
    PCG coefficients: diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j)."""
    import torch

    r = b.clone()
    z = apply_m(r)
    p = z.clone()
    rz = float(torch.dot(r, z))
    alphas, betas = [], []
    for _ in range(iters):
        q = apply_a(p)
        alpha = rz / float(torch.dot(p, q))
        r -= alpha * q
        z = apply_m(r)
        rz_new = float(torch.dot(r, z))
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1])


def pcg_elasticity_arm(args, world, rank, local):
    """Linear elasticity (lambda = mu = 1) on vector P2 tets, clamped on the face x = 0, loaded by a uniform body
    force: time to ||b - A_D u|| <= 1e-8 ||b|| for FP64 CG and Jacobi-PCG (A_D: the operator with the clamped rows and
    columns replaced by the identity)."""
    import torch

    from paper_1903_08243_gb300 import build as libbuild

    libbuild.build()
    import paper_1903_08243_gb300 as mfa

    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    ctx = mfa.Context(local, stream)
    nx = args.nx or 48
    mesh = fi.kuhn_tet_mesh(nx)
    cn, nnode, edges = fi.p2_node_map(mesh.cell_vert, mesh.nvert)
    nodes = fi.p2_node_coords(mesh.coords, edges)
    m = mfa.Mesh(ctx, mfa.MFA_CELL_TET4, mesh.coords, mesh.cell_vert)
    sp = mfa.Space(m, 2, 3, cn, nnode)
    A = mfa.Form(sp, mfa.MFA_FORM_ELASTICITY, lam=1.0, mu=1.0)
    if not args.no_autotune:  # the operator's launch configuration (setup, outside the timed solves)
        tx = torch.rand(3 * nnode, dtype=torch.float64, device="cuda")
        A.autotune(tx, torch.empty_like(tx))
        del tx
    clamped = np.flatnonzero(nodes[:, 0] < 1e-12)
    dofs = (3 * clamped[:, None] + np.arange(3)[None, :]).ravel()
    A.set_dirichlet(dofs)
    # load f_i = int b . phi_i for b = (0, 0, -1): minus the hyperelastic residual at u = 0 (P(I) = 0)
    load = mfa.Form(sp, mfa.MFA_FORM_HYPER_RES, lam=1.0, mu=1.0, b=(0.0, 0.0, -1.0))
    b = -load.apply(torch.zeros(3 * nnode, dtype=torch.float64, device="cuda"))
    b[torch.from_numpy(dofs).cuda()] = 0.0
    ctx.sync()
    rtol = 1e-8
    rows = []
    sampler = ClockSampler(local)
    sampler.start()
    for r in range(args.nrhs + 1):  # the first solve of each method warms up and is not reported
        res = {}
        for name, pc in (("cg_fp64", mfa.MFA_PC_NONE), ("jacobi_pcg_fp64", mfa.MFA_PC_JACOBI)):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, it, rel = mfa.mfa_cg(ctx.h, A.h, pc, b, x, rtol, 50000)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            true_rel = float(torch.linalg.norm(b - A.apply(x)) / torch.linalg.norm(b))
            res[name] = {"seconds": dt, "iterations": it, "relres": rel, "true_relres": true_rel, "status": rc,
                         "ms_per_iteration": dt * 1e3 / max(it, 1)}
        if r > 0:
            rows.append(res)
    clocks = sampler.stop()
    tc = statistics.mean(r["cg_fp64"]["seconds"] for r in rows)
    tj = statistics.mean(r["jacobi_pcg_fp64"]["seconds"] for r in rows)
    if rank == 0:
        line = {
            "metric": "PCG time-to-1e-8", "value": tj, "unit": "s", "n_gpus": world, "steps": args.nrhs,
            "warmup": 1, "ms_per_step": tj * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "pcg-elasticity-tet-kuhn%d^3x6-P2vec-clamped" % nx, "ndof": 3 * nnode,
                       "constrained_dofs": int(dofs.size), "lambda": 1.0, "mu": 1.0,
                       "rhs": "f_i = int b . phi_i, b = (0, 0, -1); zero at the clamped dofs",
                       "boundary": "clamped (u = 0) on the face x = 0, traction-free elsewhere",
                       "stop": "FP64 ||b - A_D u||_2 <= 1e-8 ||b||_2 from u = 0",
                       "operator": A.config().as_dict()},
            "cg_fp64_seconds": tc, "jacobi_pcg_fp64_seconds": tj, "jacobi_speedup": tc / tj, "solves": rows,
            "clocks": clocks, "roofline": None, "cpu_baseline": None, "e2e": None,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.precision is None:
        args.precision = "fp32" if args.workload == "batched" else "fp64"
    if args.degrees is None:
        args.degrees = {"hex-vector": "1,2,3,4", "tet-pk": "3,4,5,6", "planar": "1,2,3,4"}.get(args.workload,
                                                                                                "1,2,3,4,5,6")
    if args.forms is None:
        args.forms = {"hex-vector": "elasticity,hyper_res,hyper_jac", "tet-pk": "helmholtz,elasticity",
                      "planar": "helmholtz,elasticity"}.get(args.workload, "laplace,helmholtz")
    world, rank, local = dist_setup(args)
    if args.workload == "batched" and args.impl != "reference":
        batched_arm(args, world, rank, local)
    elif args.workload == "pcg" and args.impl != "reference":
        pcg_arm(args, world, rank, local)
    elif args.workload == "pcg-elasticity" and args.impl != "reference":
        pcg_elasticity_arm(args, world, rank, local)
    elif args.impl == "reference":
        reference_arm(args, world, rank)
    elif args.workload == "hex" and world > 1 and args.parallelism != "replicas":
        sharded_hex_arm(args, world, rank, local)
    else:
        gpu_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
