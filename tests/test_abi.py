"""The C-ABI library builds, loads and exports every symbol of include/rpba.h (no GPU)."""

import ctypes
import os
import re

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


def test_struct_layouts_match_header():
    # pointer-sized fields at the end of rpba_options: ctypes and C agree on size
    assert ctypes.sizeof(rpba.Options) % 8 == 0
    assert ctypes.sizeof(rpba.Problem) == 3 * 4 + 4 + 9 * 8
    assert ctypes.sizeof(rpba.Report) == 3 * 8 + 7 * 4 + 4 + 128 * 8


def test_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1910_08138_gb300 import synth
    with pytest.raises(rpba.RpbaError):
        rpba.Rpba(synth.tiny())
