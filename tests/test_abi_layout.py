"""The Python binding's ctypes structures and constants against the C header.

A small C program compiled with the host compiler against include/csff.h
prints every structure's size and field offsets and the values of the enums
and macros the binding mirrors; each must equal what the binding declares (a
mismatch would silently corrupt the arguments of every call).  CPU only."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__ as g
    g._build_module().build()
    import paper_1211_4461_gb300 as csff
    return csff


def _structs(csff):
    return {"csff_gauss": csff.Gauss, "csff_problem": csff.ProblemC, "csff_opts": csff.OptsC,
            "csff_info": csff.InfoC, "csff_plan_desc": csff.DescC, "csff_prof_stats": csff.ProfStatsC}


def _constants(csff):
    c = {"CSFF_OK": csff.OK, "CSFF_ERR_INVALID_ARG": csff.ERR_INVALID_ARG, "CSFF_ERR_CUDA": csff.ERR_CUDA,
         "CSFF_ERR_OOM": csff.ERR_OOM, "CSFF_ERR_NOT_CONVERGED": csff.ERR_NOT_CONVERGED,
         "CSFF_ERR_DIVERGED": csff.ERR_DIVERGED, "CSFF_ERR_NONFINITE": csff.ERR_NONFINITE,
         "CSFF_ERR_TIMEOUT": csff.ERR_TIMEOUT, "CSFF_ERR_UNSUPPORTED": csff.ERR_UNSUPPORTED,
         "CSFF_WARN_ILL_CONDITIONED": csff.WARN_ILL_CONDITIONED,
         "CSFF_SMOOTHER_JACOBI": csff.SMOOTHER["jacobi"], "CSFF_SMOOTHER_RBGS": csff.SMOOTHER["rbgs"],
         "CSFF_SMOOTHER_GMRES": csff.SMOOTHER["gmres"],
         "CSFF_PREC_FP64": csff.PRECISION["fp64"], "CSFF_PREC_MIXED": csff.PRECISION["mixed"],
         "CSFF_MAX_HISTORY": csff.MAX_HISTORY,
         "CSFF_FF_FP64": csff.FF_FP64, "CSFF_FF_TC_BF16X4": csff.FF_TC_BF16X4,
         "CSFF_PROF_FF_CONTRACT": csff.PROF_FF_CONTRACT, "CSFF_PROF_MG32": csff.PROF_MG32,
         "CSFF_PROF_MG64": csff.PROF_MG64, "CSFF_PROF_FF_OTHER": csff.PROF_FF_OTHER,
         "CSFF_PROF_TILES32": csff.PROF_TILES32, "CSFF_PROF_TILES32_FINE": csff.PROF_TILES32_FINE,
         "CSFF_PROF_FAMILIES": len(csff.PROF_NAMES)}
    return c


def _layout_program(structs, constants):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "csff.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("S {cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("F {cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    for name in constants:
        lines.append(f'  printf("C {name} %lld\\n", (long long)({name}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


def test_struct_layouts_and_constants_match_the_header(binding, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    structs, constants = _structs(binding), _constants(binding)
    src = tmp_path / "layout.c"
    src.write_text(_layout_program(structs, constants))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        kind, name, value = line.split()
        got[(kind, name)] = int(value)
    for cname, py in structs.items():
        assert got[("S", cname)] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[("F", f"{cname}.{fname}")] == getattr(py, fname).offset, f"{cname}.{fname}"
    for name, value in constants.items():
        assert got[("C", name)] == value, name
