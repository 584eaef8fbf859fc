"""The C ABI library loads and exports every entry point include/ljoin.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ljoin.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rmi_build", "rmi_free", "rmi_stats", "rmi_export", "join_count",
                     "join_emit", "join_host", "lj_last_error", "lj_version"):
        assert required in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2111_08824_gb300 import _native
    lib_path = _native.library_path()
    if not os.path.exists(lib_path):
        from paper_2111_08824_gb300 import build
        build.build()
    lib = ctypes.CDLL(lib_path)
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in ljoin.h but not exported"
    # the binding knows every declared function too
    assert set(_declared_functions()) <= set(_native.SIGNATURES)
    assert _native.lj_version().startswith("ljoin-gb300")


def test_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    import paper_2111_08824_gb300 as lj
    with pytest.raises(TypeError):
        lj.rmi_build(torch.zeros(4, dtype=torch.int64), 4)
