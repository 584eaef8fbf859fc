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


def test_options_are_validated_without_a_gpu():
    """Process-wide options round-trip and reject out-of-range values (host
    state only: no device call is made)."""
    import paper_2111_08824_gb300 as lj
    saved = {k: lj.lj_get_option(k) for k in ("single_pass_max", "host_chunk", "probe_buckets",
                                              "lookback_polls", "fault_skip_tiles", "fused_max",
                                              "fused_groups", "key_levels")}
    try:
        for v in (0, 1, 2):
            lj.lj_set_option("probe_buckets", v)
            assert lj.lj_get_option("probe_buckets") == v
        lj.lj_set_option("host_chunk", 1 << 20)
        assert lj.lj_get_option("host_chunk") == 1 << 20
        lj.lj_set_option("single_pass_max", 12345)
        assert lj.lj_get_option("single_pass_max") == 12345
        assert lj.lj_get_option("fused_max") == 1 << 21          # defaults
        assert lj.lj_get_option("fused_groups") == 1
        lj.lj_set_option("fused_max", 0)
        assert lj.lj_get_option("fused_max") == 0
        lj.lj_set_option("fused_groups", 0)
        assert lj.lj_get_option("fused_groups") == 0
        assert lj.lj_get_option("key_levels") == 2               # default: R with duplicates
        for v in (0, 1, 2):
            lj.lj_set_option("key_levels", v)
            assert lj.lj_get_option("key_levels") == v
        assert lj.lj_get_option("lookback_polls") == 1 << 20      # default bound
        assert lj.lj_get_option("fault_skip_tiles") == 0          # no fault injected
        lj.lj_set_option("lookback_polls", 256)
        assert lj.lj_get_option("lookback_polls") == 256
        lj.lj_set_option("fault_skip_tiles", 3)
        assert lj.lj_get_option("fault_skip_tiles") == 3
        for name, bad in (("probe_buckets", 3), ("probe_buckets", -1), ("host_chunk", 100),
                          ("host_chunk", 1 << 33), ("single_pass_max", -1), ("no_such_option", 1),
                          ("lookback_polls", 15), ("lookback_polls", (1 << 20) + 1),
                          ("fault_skip_tiles", -1), ("fault_skip_tiles", 1025),
                          ("fused_max", (1 << 22) + 1), ("fused_max", -1), ("fused_groups", 2),
                          ("key_levels", 3), ("key_levels", -1)):
            with pytest.raises(lj.LJoinError) as e:
                lj.lj_set_option(name, bad)
            assert e.value.code == -1
        with pytest.raises(lj.LJoinError):
            lj.lj_get_option("no_such_option")
    finally:
        for k, v in saved.items():
            lj.lj_set_option(k, v)


def test_null_arguments_are_rejected_without_a_gpu():
    """Entry points check their arguments before touching the device."""
    from paper_2111_08824_gb300 import _native
    lib = _native.load()
    assert lib.grmi_build(None, 4, None) == -1
    assert lib.lhash_build(None, 4, None) == -1
    assert lib.grmi_drop(None) == -1
    assert lib.grmi_stats(None, None) == -1
    assert lib.index_autotune(None, None, 0, None, None, None) == -1
    assert lib.join_expand(None, None, 0, None, 0, None, None, None) == -1
    assert lib.join_host(None, None, 0, None, 0, None, None) == -1
    assert b"NULL" in lib.lj_last_error() or b"null" in lib.lj_last_error().lower()
