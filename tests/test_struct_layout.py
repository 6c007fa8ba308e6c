"""The Python binding's ctypes structures against the C header's layout (CPU only).

A C program built with the host compiler from include/sem.h prints sizeof and offsetof for every
field of the four structures that cross the boundary; the binding's ctypes mirrors must agree,
field by field, or a call would read its arguments from the wrong bytes."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1403_0968_gb300 as sem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"sem_desc": sem.SemDesc, "sem_info": sem.SemInfo, "sem_pcg_opts": sem.SemPcgOpts,
           "sem_pcg_result": sem.SemPcgResult}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_ctypes_structures_match_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sem.h"', 'int main(void) {']
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ['  return 0;', '}']
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, py in STRUCTS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
