"""The C-ABI library loads and exports every entry point its header declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "mfa.h")).read()
    return sorted(set(re.findall(r"^MFA_API\s+[\w\s\*]*?\b(mfa_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ["mfa_create", "mfa_mesh_upload", "mfa_space_create", "mfa_form_create", "mfa_apply",
                 "mfa_apply_host", "mfa_diagonal", "mfa_cg", "mfa_sync", "mfa_last_error"]:
        assert name in syms


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1903_08243_gb300 import build as b

    path = b.build()
    import paper_1903_08243_gb300 as mfa

    L = mfa.lib()
    for name in header_symbols():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mfa_\w+)", out))
    assert set(header_symbols()) <= exported
    assert L.mfa_version() == 1


def test_binding_declares_every_symbol():
    import paper_1903_08243_gb300 as mfa

    assert set(header_symbols()) == set(mfa._SIGS)


def test_status_without_gpu_is_an_error_not_a_crash():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1903_08243_gb300 as mfa

    with pytest.raises(mfa.MfaError) as e:
        mfa.mfa_create(0, 0)
    assert e.value.code == mfa.MFA_ERR_CUDA
    assert mfa.lib().mfa_last_error()
