"""The ctypes mirrors of the C ABI's structs (paper_2602_08097_gb300) have the
same size and field offsets as the structs include/rp.h declares, as a C
compiler lays them out (gcc on the host; no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["rp_stats_t", "rp_request_info", "rp_server_stats_t", "rp_executor", "rp_server_config"]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import paper_2602_08097_gb300 as rp
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rp.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(rp, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True)
    table = {}
    for ln in out.splitlines():
        name, field, value = ln.split()
        table[(name, field)] = int(value)
    return table


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_matches_the_header(c_layout, name):
    import paper_2602_08097_gb300 as rp
    cls = getattr(rp, name)
    assert ctypes.sizeof(cls) == c_layout[(name, "size")], name
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(name, field)], (name, field)
