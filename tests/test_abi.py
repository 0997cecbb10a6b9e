"""The C-ABI library builds, loads and exports every function include/duquad.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dq_[a-z_0-9]+)\s*\(", src, re.M))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("dq_context_create", "dq_problem_create", "dq_solve", "dq_solve_many", "dq_submit",
                 "dq_poll", "dq_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1504_05708_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    lib.dq_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.dq_version()


def test_binding_lists_every_declared_symbol():
    from paper_1504_05708_gb300 import duquad
    assert _declared() <= set(duquad.SYMBOLS)


def test_oracle_and_product_share_no_code():
    """The oracle and the CUDA path import nothing from each other."""
    pkg = os.path.join(ROOT, "paper_1504_05708_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from|#include)\s+[\"<]?([a-z_]+)", src), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1504_05708_gb300" not in src and "duquad.h" not in src, f
