"""The C ABI: header declarations, exported symbols, build (CPU only)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bh.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(bh_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_02289_gb300 import _build
    if not _build.up_to_date() and shutil.which("nvcc") is None:
        pytest.skip("nvcc not available to build libbh.so")
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_path():
    names = _declared()
    for need in ("bh_create", "bh_build_tree", "bh_make_lists", "bh_compute_forces", "bh_step", "bh_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1907_02289_gb300 import bh
    assert set(bh.SYMBOLS) == set(_declared())


def test_binding_struct_layout_matches_header():
    from paper_1907_02289_gb300 import bh
    assert ctypes.sizeof(bh.bh_params) == 8 * 8 + 6 * 4 + 8
    assert ctypes.sizeof(bh.bh_particles) == 11 * 8 + 8
    assert ctypes.sizeof(bh.bh_counters) == 7 * 8


def test_load_fails_loudly_when_missing(tmp_path):
    from paper_1907_02289_gb300 import bh
    saved = bh._lib
    bh._lib = None
    try:
        with pytest.raises(RuntimeError):
            bh.load(str(tmp_path / "libbh.so"))
    finally:
        bh._lib = saved
