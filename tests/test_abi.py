"""The C-ABI library loads and exports every entry point include/mpcd.h declares
(no compute call: this runs without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_14307_gb300 import binding, build_lib
    build_lib.build()
    return binding.load()


def declared():
    hdr = open(os.path.join(ROOT, "include", "mpcd.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(mpcd_[a-z_]+)\s*\(", hdr)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for must in ("mpcd_create", "mpcd_stream", "mpcd_collide", "mpcd_couple", "mpcd_step",
                 "mpcd_destroy", "mpcd_set_state", "mpcd_get_state", "mpcd_diagnostics"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2604_14307_gb300 import binding, build_lib
    out = subprocess.run(["nm", "-D", "--defined-only", build_lib.LIB], capture_output=True,
                         text=True, check=True).stdout
    syms = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared():
        assert name in syms, name
        assert hasattr(lib, name)
    assert sorted(binding.EXPORTS) == declared()


def test_null_and_invalid_arguments_fail_cleanly(lib):
    from paper_2604_14307_gb300 import binding as B
    assert lib.mpcd_destroy(None) == B.MPCD_OK
    assert lib.mpcd_step(None, 1, None) == B.MPCD_ERR_ARG
    assert lib.mpcd_sizes(None, None) == B.MPCD_ERR_ARG
    out = C.c_void_p()
    # invalid parameters are rejected before any device call
    prm = B.Params(-1.0, 0.1, 130.0, 1.0, 0, 0, 1, 0, 1, 0, 0)
    assert lib.mpcd_create(C.byref(prm), 0, None, 1, None, None, 0, C.byref(out)) == B.MPCD_ERR_ARG
    prm = B.Params(1.0, 0.1, 130.0, 1.0, 7, 0, 1, 0, 1, 0, 0)
    assert lib.mpcd_create(C.byref(prm), 0, None, 0, None, None, 0, C.byref(out)) == B.MPCD_ERR_ARG
    assert lib.mpcd_last_error(None) == b"null context"


def test_package_import_loads_nothing():
    import importlib
    import sys
    for m in [m for m in sys.modules if m.startswith("paper_2604_14307_gb300")]:
        del sys.modules[m]
    pkg = importlib.import_module("paper_2604_14307_gb300")
    assert "paper_2604_14307_gb300.binding" not in sys.modules or pkg is not None
