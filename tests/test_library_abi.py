"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads, and
exports every entry point include/cpr.h declares (no GPU call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cpr_\w+)\s*\(", text, re.M):
                names.add(m.group(1))
    return names


def test_build_and_exports():
    from paper_2201_01970_b300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert {"cpr_setup", "cpr_update", "cpr_solve", "cpr_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_loads_and_defaults():
    import paper_2201_01970_b300 as cpr
    o = cpr.default_opts()
    assert (o.theta_color, o.theta_amg, o.mu, o.restart, o.coarse_max) == (0.05, 0.25, 30, 30, 256)
    # the fields after the stream pointer: a layout mismatch with cpr_opts would misread them
    assert (o.max_restarts, o.decouple, o.pre, o.post, o.max_levels, o.seed) == (100, 1, 1, 1, 20, 0)
    assert (o.pdl, o.tail, o.bilu_order, o.reuse_refresh, o.resetup) == (1, 0, 0, 0, 0)
    assert (o.amg, o.amli_iters, o.coloring, o.coloring_rows) == (0, 2, 0, 4096)
    assert ctypes.sizeof(cpr.Opts) == 112   # sizeof(cpr_opts), asserted at compile time in api.cu
    assert cpr.lib().cpr_strerror(cpr.CPR_ERR_SINGULAR).startswith(b"singular")


def test_oracle_header_says_test_infrastructure():
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "TEST INFRASTRUCTURE ONLY" in src
    pkg = os.path.join(ROOT, "paper_2201_01970_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert "oracle" not in open(os.path.join(dirpath, f)).read().lower(), f
