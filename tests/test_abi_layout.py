"""The ctypes mirrors of the C ABI structs have the header's exact layout (CPU).

A C program compiled against include/turtle.h prints offsetof and sizeof for every field the
Python binding declares; each must equal the ctypes field's offset and the struct's size, so a
field added, dropped or reordered on one side only fails here rather than corrupting a call.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MIRRORS = [  # (C type, Python class name in the package)
    ("turtle_params", "Params"),
    ("turtle_reads", "_Reads"),
    ("turtle_result", "_Result"),
    ("turtle_device_result", "_DeviceResult"),
    ("turtle_stats", "Stats"),
    ("turtle_job", "_Job"),
    ("turtle_job_times", "JobTimes"),
    ("turtle_server_stats", "ServerStats"),
]


def test_struct_layouts_match_the_header(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    import paper_1305_1861_gb300 as pkg

    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "turtle.h"', "int main(void) {"]
    expect = {}
    for ctype, pyname in MIRRORS:
        cls = getattr(pkg, pyname)
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (ctype, ctype))
        expect[(ctype, "sizeof")] = ctypes.sizeof(cls)
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (ctype, field, ctype, field))
            expect[(ctype, field)] = getattr(cls, field).offset
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            ctype, field, value = line.split()
            got[(ctype, field)] = int(value)
    assert got == expect
