"""The C ABI library builds, loads and exports every entry point of include/tlr.h,
and the Python binding's structures match the C layouts (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2402_09356_gb300 as tlr
from paper_2402_09356_gb300 import build as tlr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tlr.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(tlr_[a-z_0-9]+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    tlr_build.build()
    return tlr.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", tlr.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in nm.splitlines() if " T " in l)
    assert set(names) <= exported
    assert sorted(tlr.exported_symbols()) == names


def test_version_without_gpu(lib):
    assert tlr.tlr_version().startswith("tlr-gb300")
    assert tlr.tlr_tiles_size(1600, 200) == 36 * 200 * 200
    assert tlr.tlr_tiles_size(1001, 100) == 66 * 100 * 100


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "lay.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "tlr.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(tlr_theta), sizeof(tlr_opts), sizeof(tlr_result), sizeof(tlr_pool_opts));
  printf("%zu %zu %zu %zu\\n", offsetof(tlr_opts, eps), offsetof(tlr_opts, precision),
         offsetof(tlr_result, info), offsetof(tlr_result, ms_total));
  printf("%zu %zu %zu\\n", offsetof(tlr_pool_opts, hbm_budget), offsetof(tlr_result, precision_used),
         offsetof(tlr_result, min_pivot2));
  return 0;
}
""")
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:4] == [ctypes.sizeof(tlr.tlr_theta), ctypes.sizeof(tlr.tlr_opts), ctypes.sizeof(tlr.tlr_result),
                         ctypes.sizeof(tlr.tlr_pool_opts)]
    assert sizes[4:] == [tlr.tlr_opts.eps.offset, tlr.tlr_opts.precision.offset, tlr.tlr_result.info.offset,
                         tlr.tlr_result.ms_total.offset, tlr.tlr_pool_opts.hbm_budget.offset,
                         tlr.tlr_result.precision_used.offset, tlr.tlr_result.min_pivot2.offset]


def test_context_creation_fails_cleanly_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tlr.TlrError):
        tlr.Context(0)
