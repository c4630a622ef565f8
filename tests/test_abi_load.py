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


def header_enums():
    txt = open(os.path.join(ROOT, "include", "mfa.h")).read()
    return {k: int(v) for k, v in re.findall(r"\b(MFA_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}


def test_binding_constants_match_the_header():
    import ctypes

    import paper_1903_08243_gb300 as mfa

    enums = header_enums()
    checked = 0
    for name, value in enums.items():
        if hasattr(mfa, name):
            assert getattr(mfa, name) == value, name
            checked += 1
    assert checked >= 30
    for name in ["MFA_VARIANT_POINT", "MFA_VARIANT_EVEN_ODD", "MFA_VARIANT_LINE", "MFA_VARIANT_LINE_STAGED",
                 "MFA_VARIANT_CELL"]:
        assert getattr(mfa, name) == enums[name]


def test_binding_structs_have_the_header_layout(tmp_path):
    """sizeof/offsetof of every struct the binding mirrors, as the C compiler lays it out from the header."""
    import ctypes

    import paper_1903_08243_gb300 as mfa

    structs = {"mfa_form_params": mfa.mfa_form_params, "mfa_form_info": mfa.mfa_form_info,
               "mfa_launch_config": mfa.mfa_launch_config}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mfa.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(r'printf("%s %%zu\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            cfield = {"lam": "lambda"}.get(field, field)  # `lambda` is a Python keyword
            lines.append(r'printf("%s.%s %%zu\n", offsetof(%s, %s));' % (name, field, name, cfield))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[name + "." + field]) == getattr(cls, field).offset, (name, field)
