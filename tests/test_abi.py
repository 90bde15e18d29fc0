"""The C-ABI library builds, loads and exports every entry point of include/gf.h (CPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:gf_status|const char\s*\*)\s*(gf_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("gf_create", "gf_load_field", "gf_build_bvh", "gf_set_lod_mask",
                     "gf_transmittance", "gf_render", "gf_render_backward", "gf_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2602_05081_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(gf_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_wraps_every_symbol():
    from paper_2602_05081_gb300 import _abi
    for n in _declared():
        assert n in _abi.EXPORTED, n
        assert hasattr(_abi, n), n


def test_create_without_gpu_fails_cleanly():
    """No GPU here: gf_create reports an error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2602_05081_gb300 import _abi
    with pytest.raises(_abi.GfError):
        _abi.gf_create(0)
