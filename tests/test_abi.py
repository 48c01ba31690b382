"""The C-ABI library builds, loads and exports every entry point that include/tt_iga.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tt_iga.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(tt_iga_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as g
    g.build()
    return os.path.join(ROOT, "paper_2509_13224_gb300", "libtt_iga.so")


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ["tt_iga_ctx_create", "tt_iga_geometry", "tt_iga_assemble", "tt_iga_solve", "tt_iga_eval",
                     "tt_iga_l2_error", "tt_iga_densify_operator", "tt_iga_round", "tt_iga_stiffness_core"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(lib_path):
    import paper_2509_13224_gb300 as tt
    assert sorted(tt.exported_symbols()) == declared_functions()


def test_struct_layouts_match_header(lib_path, tmp_path):
    """sizeof/offsetof from a C compiler reading include/tt_iga.h equal the ctypes mirror."""
    import subprocess
    import paper_2509_13224_gb300 as tt
    structs = {"tt_iga_geom_desc": tt.GeomDesc, "tt_iga_rhs_desc": tt.RhsDesc, "tt_iga_solve_opts": tt.SolveOpts,
               "tt_iga_stats": tt.Stats, "tt_iga_ctx_opts": tt.CtxOpts, "tt_iga_batch_item": tt.BatchItem,
               "tt_iga_bc_desc": tt.BcDesc, "tt_iga_nurbs_patch": tt.NurbsPatch,
               "tt_iga_batch_result": tt.BatchResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tt_iga.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            c, f, v = line.split()
            got[(c, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)


def test_launch_counter_without_gpu(lib_path):
    import paper_2509_13224_gb300 as tt
    assert tt.tt_iga_launch_count() >= 0


def test_context_creation_fails_cleanly_without_gpu(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2509_13224_gb300 as tt
    with pytest.raises(tt.TTIgaError):
        tt.tt_iga_ctx_create()
