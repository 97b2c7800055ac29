"""The binding's ctypes structures against the C header: a small C program
compiled against include/ep.h prints the size of every struct the binding
mirrors and the offset of each of its fields, which must equal what ctypes
lays out (a field added on one side only, or in another order, would pass
garbage through the C ABI without an error)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2308_01651_gb300 import ep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [ep.ep_mesh, ep.ep_fibers, ep.ep_conductivities, ep.ep_ionic_model, ep.ep_pulse, ep.ep_stimulus,
           ep.ep_options, ep.ep_stats, ep.ep_kernel_time]


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ep.h"', "int main(void) {"]
    for S in STRUCTS:
        n = S.__name__
        lines.append(f'    printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _ in S._fields_:
            lines.append(f'    printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        name, field, value = line.split()
        table[(name, field)] = int(value)
    return table


def test_ctypes_structures_match_the_header(tmp_path):
    table = c_layout(tmp_path)
    for S in STRUCTS:
        n = S.__name__
        assert table[(n, "sizeof")] == C.sizeof(S), n
        for f, _ in S._fields_:
            assert table[(n, f)] == getattr(S, f).offset, (n, f)
