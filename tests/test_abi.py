"""The C-ABI library loads and exports every entry point include/*.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(rkhsba_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2403_01254_gb300 import _build
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rkhsba_create", "rkhsba_eval", "rkhsba_solve", "rkhsba_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    import paper_2403_01254_gb300 as pk
    assert set(pk.EXPORTS) <= set(_declared())
    for n in pk.EXPORTS:
        if n not in ("rkhsba_last_error",):
            assert hasattr(pk.rkhsba, n) or n in ("rkhsba_create_device",)


def test_launch_counter_and_error_string_without_gpu(lib):
    lib.rkhsba_launch_count.restype = ctypes.c_int64
    lib.rkhsba_last_error.restype = ctypes.c_char_p
    lib.rkhsba_last_error.argtypes = [ctypes.c_void_p]
    assert lib.rkhsba_launch_count() >= 0
    assert isinstance(lib.rkhsba_last_error(None), bytes)


def test_built_for_sm_103a_only():
    from paper_2403_01254_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_does_not_reach_the_oracle():
    pkg = os.path.join(ROOT, "paper_2403_01254_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h")):
            txt = open(path).read()
            assert "import oracle" not in txt and "from oracle" not in txt, path
