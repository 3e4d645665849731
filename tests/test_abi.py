"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/percis.h declares; the binding's signature table matches the
header.  No compute calls (they need a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "percis.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(percis_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_11454_gb300 import build_lib

    path = build_lib.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2509_11454_gb300 import binding

    assert sorted(binding.SIGNATURES) == _declared()


def test_binding_loads_and_reports_without_gpu(lib):
    from paper_2509_11454_gb300 import binding

    binding.load_library()
    opt = binding.percis_default_options()
    assert opt.form == binding.FORM_BATCHED and opt.keep_paths == 1 and opt.vertex_diam == -1
    assert opt.timeout_s == 10.0


def test_struct_layouts_match_header():
    """Field order and sizes of the ctypes mirrors against a C compile of the header."""
    import subprocess
    import tempfile

    from paper_2509_11454_gb300 import binding

    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "percis.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(percis_options), offsetof(percis_options, timeout_s),
         sizeof(percis_info), offsetof(percis_info, kernel_launches));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(binding.percis_options)
    assert vals[1] == binding.percis_options.timeout_s.offset
    assert vals[2] == ctypes.sizeof(binding.percis_info)
    assert vals[3] == binding.percis_info.kernel_launches.offset
