"""The C-ABI library loads and exports every entry point that include/hotrg.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hotrg.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hotrg_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_20536_b300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hotrg_create", "hotrg_destroy", "hotrg_init_tensor", "hotrg_step", "hotrg_run",
                     "hotrg_observables", "hotrg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        getattr(lib, f)


def test_struct_layout_matches_header():
    from paper_2609_20536_b300 import hotrg as H
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "hotrg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(hotrg_params), sizeof(hotrg_step_info), sizeof(hotrg_result),
         sizeof(hotrg_obs), offsetof(hotrg_result, step), offsetof(hotrg_params, tie_rtol),
         sizeof(hotrg_scaling), offsetof(hotrg_scaling, y_std));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = list(map(int, subprocess.check_output([exe]).split()))
    assert got == [ctypes.sizeof(H.Params), ctypes.sizeof(H.StepInfo), ctypes.sizeof(H.Result),
                   ctypes.sizeof(H.Obs), H.Result.step.offset, H.Params.tie_rtol.offset,
                   ctypes.sizeof(H.Scaling), H.Scaling.y_std.offset]


def test_no_device_call_without_gpu(lib):
    # version string needs no device
    lib.hotrg_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hotrg_version()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_20536_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
