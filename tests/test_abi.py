"""The C-ABI library builds, loads and exports every entry point of include/gf.h (CPU)."""
import ctypes as C
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


def test_header_declares_the_caller_allocator():
    """Device memory of the library comes from a caller-supplied allocator: the
    header declares the callback struct (alloc and free, with the stream), the
    context constructor that takes it, and the reserve call that sizes the
    compute calls' scratch ahead."""
    src = open(os.path.join(ROOT, "include", "gf.h")).read()
    assert re.search(r"void\*\s*\(\*alloc\)\(void\*\s*user,\s*size_t\s*bytes,\s*gf_stream\s*stream\)", src)
    assert re.search(r"void\s*\(\*free\)\(void\*\s*user,\s*void\*\s*ptr,\s*size_t\s*bytes,\s*gf_stream\s*stream\)",
                     src)
    names = _declared()
    assert "gf_create_ex" in names and "gf_reserve" in names


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


def _c_layout(header_dir, header, structs, tmp_path):
    """sizeof and offsetof of every field, as a C compiler lays the structs out."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "%s"' % header, "int main(void) {"]
    for cname, pyname, fields in structs:
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (pyname, cname))
        for f in fields:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (pyname, f, cname, f))
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", header_dir, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.split("\n"):
        if ln:
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    return got


def _check(structs, got):
    for _, py, fields in structs:
        assert got[(py.__name__, "size")] == C.sizeof(py), py.__name__
        for f in fields:
            assert got[(py.__name__, f)] == getattr(py, f).offset, (py.__name__, f)



def test_binding_structs_match_the_c_layout(tmp_path):
    """Every ctypes mirror of an include/gf.h struct has the C compiler's size and
    field offsets (the structs are passed by pointer through the C ABI)."""
    from paper_2602_05081_gb300 import _abi
    pys = [_abi.gf_params, _abi.gf_field_opts, _abi.gf_lod_desc, _abi.gf_camera,
           _abi.gf_render_opts, _abi.gf_stats, _abi.gf_server_opts, _abi.gf_request,
           _abi.gf_result, _abi.gf_server_stats, _abi.gf_allocator, _abi.gf_reserve_opts]
    structs = [(py.__name__, py, [f for f, _ in py._fields_]) for py in pys]
    got = _c_layout(os.path.join(ROOT, "include"), "gf.h",
                    [(c, py.__name__, fs) for c, py, fs in structs], tmp_path)
    _check(structs, got)


def test_oracle_structs_match_the_c_layout(tmp_path):
    """The same for the oracle's ctypes mirrors of oracle/gf_oracle.h."""
    import oracle
    pairs = [("or_field_desc", oracle.FieldDesc), ("or_lod", oracle.Lod),
             ("or_camera", oracle.Camera), ("or_render_opts", oracle.RenderOpts)]
    structs = [(c, py, [f for f, _ in py._fields_]) for c, py in pairs]
    got = _c_layout(os.path.join(ROOT, "oracle"), "gf_oracle.h",
                    [(c, py.__name__, fs) for c, py, fs in structs], tmp_path)
    _check(structs, got)
