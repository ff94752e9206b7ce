"""The C-ABI library loads and exports every entry point include/to.h declares,
and the ctypes structs match the C layouts.  No GPU work: no compute call is
made (to_default_params and to_last_error touch host memory only)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "to.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2204_06204_gb300 import _abi, _build
    _build.build()
    return _abi.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(to_[a-z_A-Z0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2204_06204_gb300 import _abi
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert n in _abi.SIGNATURES, f"{n} missing from the binding"
    assert set(_abi.SIGNATURES) == set(names)


def test_host_only_calls(lib):
    from paper_2204_06204_gb300 import _abi
    p = _abi.to_params()
    lib.to_default_params(C.byref(p))
    assert p.precision == _abi.TO_FP32_MIXED and p.n_inner == 5 and abs(p.m - 0.75) < 1e-15
    assert isinstance(lib.to_last_error(), bytes)
    # a null problem is rejected without touching a device
    assert lib.to_sizes(None, None, None) == _abi.TO_ERR_ARG
    assert b"null" in lib.to_last_error()


def test_struct_layouts_match_c():
    from paper_2204_06204_gb300 import _abi
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "to.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(to_grid), sizeof(to_material), sizeof(to_loads),
         sizeof(to_bcs), sizeof(to_params), sizeof(to_stats));
  printf("%zu %zu %zu\n", offsetof(to_params, mg_omega), offsetof(to_params, tile_z), offsetof(to_stats, status));
  return 0;
}
"""
    tmp = os.path.join(ROOT, "paper_2204_06204_gb300", "_build")
    os.makedirs(tmp, exist_ok=True)
    src = os.path.join(tmp, "layout.c")
    exe = os.path.join(tmp, "layout")
    open(src, "w").write(prog)
    subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe])
    out = subprocess.check_output([exe]).decode().split()
    sizes = [int(v) for v in out]
    assert sizes[:6] == [C.sizeof(s) for s in (_abi.to_grid, _abi.to_material, _abi.to_loads, _abi.to_bcs,
                                                _abi.to_params, _abi.to_stats)]
    assert sizes[6] == _abi.to_params.mg_omega.offset
    assert sizes[7] == _abi.to_params.tile_z.offset
    assert sizes[8] == _abi.to_stats.status.offset


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2204_06204_gb300 import _abi
    saved = _abi._lib
    try:
        _abi._lib = None
        with pytest.raises(ImportError):
            _abi.load(str(tmp_path / "missing.so"))
    finally:
        _abi._lib = saved
