"""The ctypes binding mirrors every struct of include/subcull.h that crosses
the boundary: a C program compiled against the header prints sizeof and the
offset of each field, and they must equal ctypes' layout of the binding's
classes (a field added on one side only would shift every later field)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2305_08343_gb300 import subcull as sc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = [sc.sc_scene_params, sc.sc_ray_params, sc.sc_build_opts, sc.sc_bvh_info,
           sc.sc_wave_out, sc.sc_trace_opts, sc.sc_tune_result, sc.sc_refit_info,
           sc.sc_frontier_entry]


def _program():
    lines = ['#include "subcull.h"', "#include <stddef.h>", "#include <stdio.h>",
             "int main(void) {"]
    for cls in STRUCTS:
        name = cls.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


def test_ctypes_structs_match_the_header(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text(_program())
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, key, value = line.split()
        got[(name, key)] = int(value)
    for cls in STRUCTS:
        name = cls.__name__
        assert got[(name, "size")] == C.sizeof(cls), f"{name}: size"
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, f"{name}.{field}"
