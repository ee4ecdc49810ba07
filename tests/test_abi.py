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
    assert ctypes.sizeof(bh.bh_params) == 8 * 8 + 6 * 4 + 8 + 8
    assert ctypes.sizeof(bh.bh_particles) == 11 * 8 + 8
    assert ctypes.sizeof(bh.bh_counters) == 12 * 8 + bh.BH_N_STAGES * (8 + 8) + 3 * 8
    assert ctypes.sizeof(bh.bh_tuning) == 9 * 4


def test_load_fails_loudly_when_missing(tmp_path):
    from paper_1907_02289_gb300 import bh
    saved = bh._lib
    bh._lib = None
    try:
        with pytest.raises(RuntimeError):
            bh.load(str(tmp_path / "libbh.so"))
    finally:
        bh._lib = saved


def test_header_is_plain_c_and_struct_sizes_agree(tmp_path):
    """bh.h compiles as C99 (a C caller needs no C++), and the sizes and
    field offsets a C compiler gives the ABI structs are the binding's."""
    import subprocess
    from paper_1907_02289_gb300 import bh
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "probe.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "bh.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bh_params), sizeof(bh_particles), sizeof(bh_counters),
           sizeof(bh_tuning), sizeof(bh_diagnostics), offsetof(bh_params, n_g), offsetof(bh_params, list_capacity));
    return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(bh.bh_params), ctypes.sizeof(bh.bh_particles), ctypes.sizeof(bh.bh_counters),
            ctypes.sizeof(bh.bh_tuning), ctypes.sizeof(bh.bh_diagnostics), bh.bh_params.n_g.offset,
            bh.bh_params.list_capacity.offset]
    assert got == want
