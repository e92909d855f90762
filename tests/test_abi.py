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


def test_adaptive_refinement_schedule_host_helper(lib):
    import paper_1211_4461_gb300 as csff
    f = csff.refinement_cycles
    # rho = 0.5 per cycle: from 1e-6, 1e-8 needs log2(100) = 6.64 -> 7 cycles
    assert f(1e-6 * 2 ** 6, 1e-6, 6, 1e-8, 10) == 7
    assert f(1e-6 * 2 ** 6, 1e-6, 6, 1e-8, 6) == 6                 # clamped to the step size
    assert f(1.0, 0.1 ** 6, 6, 1e-8, 6) == 2                        # rho = 0.1: 1e-6 -> 1e-8 in 2
    assert f(1.0, 2e-8, 1, 1e-8, 6) == 1                            # one cycle is enough
    assert f(1.0, 5e-9, 3, 1e-8, 6) == 1                            # already converged: at least 1
    assert f(1e-3, 2e-3, 3, 1e-8, 6) == 6                           # no reduction: full step
    assert f(1e-3, 0.0, 3, 1e-8, 6) == 6                            # degenerate inputs: full step
    assert f(float("nan"), 1e-4, 3, 1e-8, 6) == 6
    assert f(1.0, 0.999999, 1, 1e-8, 6) == 6                        # rho near 1: capped
    assert f(1.0, 0.5, 1, 1e-8, 0) == 1                             # cap below 1 counts as 1
    # the prediction reaches the tolerance: rho^n rel_after <= rel_tol
    for rho in (0.2, 0.35, 0.5, 0.7):
        for rel in (1e-3, 3e-5, 2e-7):
            n = f(rel / rho ** 4, rel, 4, 1e-8, 1000)
            assert rel * rho ** n <= 1e-8 * (1 + 1e-12) and rel * rho ** (n - 1) > 1e-8 * (1 - 1e-12)


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
