"""The C-ABI library loads and exports every function include/psfd.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "psfd.h")).read()
    return sorted(set(re.findall(r"PSFD_API\s+[\w\s\*]+?\b((?:psfd|fno)_\w+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = header_functions()
    for n in ("psfd_plan_create", "psfd_background", "psfd_apply", "psfd_precond", "psfd_solve", "fno_forward",
              "psfd_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2607_25330_b300 import build
    lib_path = build.build()
    L = ctypes.CDLL(lib_path)
    for n in header_functions():
        assert hasattr(L, n), n


def test_binding_signatures_cover_the_header():
    from paper_2607_25330_b300 import psfd
    assert sorted(psfd.declared_symbols()) == header_functions()


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2607_25330_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f
