"""The ctypes structures of the binding have the sizes and field offsets of
the C structures in include/gwns.h (compiled here with gcc; no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "ns_prior": "_Prior", "ns_data": "_Data", "ns_psd": "_Psd", "ns_grid": "_Grid",
    "ns_options": "_Options", "ns_samples": "_Samples", "ns_stats": "_Stats",
    "ns_server_options": "_ServerOptions", "ns_request": "_Request", "ns_request_status": "_ReqStatus",
}


def c_layout(tmp_path, structs):
    """sizeof and offsetof of every field, as the C compiler lays them out."""
    import paper_2509_24949_gb300 as g
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gwns.h"', "int main(void) {"]
    for cname, pyname in structs.items():
        cls = getattr(g, pyname)
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("    return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        parts = ln.split()
        res[(parts[0], parts[1])] = int(parts[2])
    return res


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_structures_match_the_header(tmp_path):
    import paper_2509_24949_gb300 as g
    lay = c_layout(tmp_path, STRUCTS)
    for cname, pyname in STRUCTS.items():
        cls = getattr(g, pyname)
        assert ctypes.sizeof(cls) == lay[(cname, "size")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == lay[(cname, fname)], (cname, fname)
