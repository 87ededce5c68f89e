"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import subprocess

import pytest

from paper_2406_09857_gb300 import build as vxbuild
from paper_2406_09857_gb300 import vx


@pytest.fixture(scope="module")
def libpath():
    return vxbuild.build()


def test_exports_every_declared_symbol(libpath):
    declared = vx.declared_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing


def test_loads_and_answers_without_device(libpath):
    L = vx.lib()
    for name in vx.declared_symbols():
        assert hasattr(L, name)
    assert L.vx_kernel_kind_name(0).decode() == "stage0_fp64"
    assert L.vx_kernel_kind_name(99).decode() == ""
    # argument checks happen before any device work
    h = ctypes.c_void_p()
    rc = L.vx_system_create(None, 0, None, ctypes.byref(h))
    assert rc == vx.EINVAL
    assert b"polynomials" in L.vx_last_error()


def test_opts_layout_matches_header(tmp_path):
    """The binding's vx_opts and vx_poly have the header's size and field offsets, as a C
    compiler lays them out."""
    inc = vxbuild.INCLUDE
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vx.h"', "int main(void) {",
             '  printf("opts %zu\\n", sizeof(vx_opts));', '  printf("poly %zu\\n", sizeof(vx_poly));']
    for name, _ in vx.Opts._fields_:
        lines.append('  printf("%s %%zu\\n", offsetof(vx_opts, %s));' % (name, name))
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                        text=True, check=True).stdout.splitlines())
    assert int(got.pop("opts")) == ctypes.sizeof(vx.Opts)
    assert int(got.pop("poly")) == ctypes.sizeof(vx.Poly)
    for name, _ in vx.Opts._fields_:
        assert int(got[name]) == getattr(vx.Opts, name).offset, name
