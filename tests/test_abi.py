"""The C-ABI library builds, loads and exports every symbol of include/rpba.h (no GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

from paper_1910_08138_gb300 import build, rpba

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = rpba.exported_symbols()
    hdr = open(os.path.join(ROOT, "include", "rpba.h")).read()
    # every function prototype of the header is listed
    assert len(names) == len(set(re.findall(r"\b(rpba_\w+)\s*\(", hdr)))
    assert {"rpba_create", "rpba_intersect", "rpba_iterate", "rpba_covariance",
            "rpba_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_default_options_are_the_papers_values():
    o = rpba.rpba_default_options()
    assert o.lambda0 == 1e-4 and o.t_v == 4.0 and o.downweight == 1e-4
    assert o.stop_ratio == 1.01 and o.grace == 1


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of rpba_problem, rpba_options and rpba_report have
    the size and the field offsets the C compiler gives the header's structs."""
    structs = {"rpba_problem": rpba.Problem, "rpba_options": rpba.Options, "rpba_report": rpba.Report}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rpba.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'  printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])


def test_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1910_08138_gb300 import synth
    with pytest.raises(rpba.RpbaError):
        rpba.Rpba(synth.tiny())
