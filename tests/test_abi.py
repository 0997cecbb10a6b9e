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


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding marshals has the header's size and field offsets (gcc on the
    header, no GPU): a field added on one side only would shift every later field."""
    import subprocess
    from paper_1504_05708_gb300 import duquad as D
    pairs = {"dq_problem_desc": D.ProblemDesc, "dq_solve_opts": D.SolveOpts, "dq_result": D.Result,
             "dq_outputs": D.Outputs, "dq_stats": D.Stats, "dq_theory_in": D.TheoryIn,
             "dq_theory_out": D.TheoryOut, "dq_theory_solve_opts": D.TheorySolveOpts,
             "dq_sparse_desc": D.SparseDesc}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "duquad.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            cfield = "lambda" if fname == "lambda_" else fname
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {cfield}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
