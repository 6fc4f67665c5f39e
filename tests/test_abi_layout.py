"""The Python binding's ctypes structures against the C header (no GPU).

A small C program, generated from the binding's field lists, includes
include/fz.h and prints the size of every public struct and the offset of
every field; each must equal what ctypes computes.  A field renamed, added or
moved on one side only fails here (a name the header lacks does not compile).
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2407_20474_gb300 as fz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["fz_opts_t", "fz_tune_entry_t", "fz_plan_info_t", "fz_memo_info_t", "fz_instance_t",
           "fz_batch_tune_entry_t", "fz_batch_info_t", "fz_serve_cfg_t", "fz_result_t",
           "fz_serve_stats_t"]


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fz.h"', "int main(void) {"]
    expect = {}
    for name in STRUCTS:
        cls = getattr(fz, name)
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        expect[name] = ctypes.sizeof(cls)
        for field in cls._fields_:
            f = field[0]
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
            expect["%s.%s" % (name, f)] = getattr(cls, f).offset
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    assert set(got) == set(expect)
    for key, val in expect.items():
        assert int(got[key]) == val, (key, got[key], val)
