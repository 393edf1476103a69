"""The ctypes mirrors of the C-ABI structs have the C compiler's layout:
every field at the offset gcc gives it, and the same total size."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ccpm_options": "Options",
    "ccpm_counts": "Counts",
    "ccpm_constraint_log": "ConstraintLog",
    "ccpm_constraint_info": "ConstraintInfo",
    "ccpm_explore_variant": "ExploreVariant",
    "ccpm_wide_stats": "WideStats",
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_1912_08453_gb300 import ccpm
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ccpm.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in getattr(ccpm, pyname)._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        s, f, v = line.split()
        table[(s, f)] = int(v)
    return table


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout(c_layout, cname):
    from paper_1912_08453_gb300 import ccpm
    cls = getattr(ccpm, STRUCTS[cname])
    assert c_layout[(cname, "sizeof")] == ctypes_sizeof(cls)
    for f, _ in cls._fields_:
        assert c_layout[(cname, f)] == getattr(cls, f).offset, f


def ctypes_sizeof(cls):
    import ctypes
    return ctypes.sizeof(cls)
