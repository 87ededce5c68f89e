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


def test_opts_layout_matches_header():
    # vx_opts: 5 int32-sized fields + 7 reserved = 48 bytes
    assert ctypes.sizeof(vx.Opts) == 48
    assert ctypes.sizeof(vx.Poly) == 24
