"""bench.py's reference arm (the FP64 oracle on the host cores) keeps its output contract: one JSON line with the
metric, unit and direction of the GPU arm, `impl: reference`, a `cpu_baseline` describing the run and an `e2e`
object with zero copy bytes; under torchrun only rank 0 prints (checked on CPU with a small workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tet-p1-mass",
           "--steps", "2", "--warmup", "1", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return lines


def test_reference_arm_json_line():
    lines = run_reference()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "operator-action GDoF/s" and d["unit"] == "GDoF/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("tet-kuhn8^3x6-P1-mass")


@pytest.mark.skipif(sys.platform != "linux", reason="torchrun rendezvous on 127.0.0.1")
def test_reference_arm_under_torchrun_prints_once():
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--workload", "tet-p1-mass", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["n_gpus"] == 2


def test_all_cores_oracle_timing_splits_cells_exactly():
    """The all-cores CPU figure runs the unchanged oracle on disjoint cell shares in spawned processes; the
    reduced result equals one oracle apply over the whole sample."""
    import argparse
    import importlib.util

    import oracle

    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    sys.modules["bench"] = bench
    spec.loader.exec_module(bench)
    args = argparse.Namespace(workload="tet-p2", nx=3, degrees=None, forms=None, order="lex", rule="auto",
                              geometry="stored", precision="fp64")
    cases = bench.build_cases(args)
    single = bench.oracle_rate(cases, samples={("tet", 2): 100})
    for workers in (2, 3):
        allc = bench.oracle_rate_all_cores(cases, single, workers)
        for c, s, a in zip(cases, single, allc):
            cv, cn, nodes, nsub = bench.sub_mesh(c, s["sample_cells"])
            xs = c["x"].reshape(-1, c["ncomp"])[nodes].ravel()
            pb = oracle.Problem(c["cell_type"], c["mesh"].coords, cv, c["p"], cn, nodes.size,
                                bench.FORM_IDS[c["form"]], ncomp=c["ncomp"], qdeg=c["qdeg"], **c["okw"])
            ref = float(pb.apply(xs).sum())
            assert a["sample_cells"] == nsub and a["full_s"] > 0
            assert abs(a["checksum"] - ref) <= 1e-12 * max(1.0, abs(ref))
