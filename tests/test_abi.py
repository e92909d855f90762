"""The C-ABI library builds, loads and exports every symbol declared in
include/csff.h; host-side argument checks work without a GPU.  CPU only: no
call here touches the device."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(csff_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    path = g._build_module().build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("csff_plan_create", "csff_solve", "csff_far_field", "csff_residual", "csff_smooth",
                 "csff_restrict", "csff_prolong_add", "csff_coarse_solve", "csff_norm2", "csff_rhs"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (csff_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_covers_the_header(lib):
    import paper_1211_4461_gb300 as csff
    assert set(_declared()) <= set(csff.EXPORTS)


def test_gamma_from_ecs_host_helper(lib):
    import paper_1211_4461_gb300 as csff
    import math
    assert abs(math.degrees(csff.gamma_from_ecs(math.pi / 6)) - 9.9) < 0.05


@pytest.mark.parametrize("bad", [
    {"dim": 4}, {"n": 64}, {"gamma": 0.0}, {"gamma": 1.0}, {"k": -1.0}, {"hi": -10.0},
    {"gaussians": [{"amp": -0.5, "width": -2.0}]},
])
def test_plan_rejects_invalid_problem_without_touching_the_gpu(lib, bad):
    import paper_1211_4461_gb300 as csff
    import workloads as W
    c = W.small_2d()
    p = dict(c["problem"])
    p.update(bad)
    with pytest.raises(csff.CsffError) as ei:
        csff.Plan(p, c["opts"], stream=_NoStream())
    assert ei.value.status == csff.ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [{"smoother": "sor"}, {"nu1": 0, "nu2": 0}, {"coarsest_n": 9, "n": 65},
                                 {"omega": 2.5}, {"rel_tol": 0.0}])
def test_plan_rejects_invalid_options(lib, bad):
    import paper_1211_4461_gb300 as csff
    import workloads as W
    c = W.small_2d()
    o = dict(c["opts"])
    p = dict(c["problem"])
    if "n" in bad:
        p["n"] = 66
    o.update({k: v for k, v in bad.items() if k != "n"})
    with pytest.raises((csff.CsffError, KeyError)):
        csff.Plan(p, o, stream=_NoStream())


class _NoStream:
    """Stands in for a torch stream on a machine without a GPU (the plan is
    rejected before any CUDA call)."""
    cuda_stream = 0
