"""The C ABI from plain C: paper_1903_08243_gb300/examples/helmholtz_host.c compiles as C11 with warnings as errors
and links against libmfa.so (CPU); on a GPU it runs and checks sum(A 1) = |Omega| for Helmholtz with k^2 = 1."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_1903_08243_gb300")
SRC = os.path.join(PKG, "examples", "helmholtz_host.c")


def build_example(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    if not os.path.exists(os.path.join(PKG, "libmfa.so")):
        pytest.skip("libmfa.so not built")
    exe = str(tmp_path / "helmholtz_host")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
           "-L", PKG, "-lmfa", "-lm", "-Wl,-rpath," + PKG, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_example_compiles_and_links(tmp_path):
    build_example(tmp_path)


@pytest.mark.gpu
def test_example_runs(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    exe = build_example(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
