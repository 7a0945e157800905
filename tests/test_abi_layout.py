"""The Python binding's ctypes structs have the layout include/mpcd.h gives
their C counterparts: every struct's size and every field's offset, read from
a probe compiled with the host C compiler against the header (no GPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("Params", "mpcd_params"), ("ShapeDesc", "mpcd_shape_desc"), ("ReplicaDesc", "mpcd_replica_desc"),
         ("Allocator", "mpcd_allocator"), ("HostState", "mpcd_host_state"), ("Sizes", "mpcd_sizes_t"),
         ("Diag", "mpcd_diag"), ("KernelTime", "mpcd_kernel_time"), ("Rnemd", "mpcd_rnemd"),
         ("Tuning", "mpcd_tuning")]


def test_ctypes_structs_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2604_14307_gb300 import binding as B
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpcd.h"', "int main(void) {"]
    expect = {}
    for py, c in PAIRS:
        cls = getattr(B, py)
        lines.append(f'printf("{c} size %zu\\n", sizeof({c}));')
        expect[f"{c} size"] = ctypes.sizeof(cls)
        for name, _ in cls._fields_:
            lines.append(f'printf("{c} {name} %zu\\n", offsetof({c}, {name}));')
            expect[f"{c} {name}"] = getattr(cls, name).offset
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        key, val = ln.rsplit(" ", 1)
        got[key] = int(val)
    assert got == expect
