"""Full multigrid (Sec. 4, FMG paragraph; Table 3) through the C ABI against
the oracle's nested iteration: the V-cycles run on every level, the finest
level's residual history and the solution.  GPU only."""
import numpy as np
import pytest

import oracle.csff_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4461_gb300 as m
    return m


def _cases():
    c2 = W.mixed_2d(5.0, n=129)
    c2["opts"].update(precision="fp64", coarsest_n=5, rel_tol=1e-9)
    c2["name"] = "2d-n129-rbgs"
    cj = W.small_2d(n=65)
    cj["name"] = "2d-n65-jacobi"
    c3 = W.paper_gmres(dim=3, k=1.0, n=33)
    c3["opts"].update(precision="fp64")
    c3["name"] = "3d-n33-gmres3-table3"
    return [c2, cj, c3]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_fmg_matches_oracle_nested_iteration(csff, case):
    plan = csff.Plan(case["problem"], case["opts"])
    p = O.problem_from_dict(case["problem"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info, cyc = plan.solve_fmg(case["eta"], u)
    assert st == csff.OK
    ref = O.fmg_solve(p, O.rhs(p, case["eta"][0]), O.opts_from_dict(case["opts"]))
    assert cyc[0] == ref.level_cycles
    assert info[0]["cycles"] == ref.cycles
    np.testing.assert_allclose(info[0]["history"], ref.history, rtol=1e-6, atol=1e-15)
    ug = u.cpu().numpy().reshape(ref.u.shape)
    assert np.linalg.norm(ug - ref.u) <= 1e-8 * np.linalg.norm(ref.u)
    plan.close()


def test_fmg_needs_an_fp64_plan(csff):
    c = W.mixed_2d(5.0, n=65)
    c["opts"].update(precision="mixed", coarsest_n=5)
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    with pytest.raises(csff.CsffError):
        plan.solve_fmg(c["eta"], u)
    plan.close()


def test_fmg_finest_cycles_against_table3_on_256(csff):
    """Table 3's setting on the 256^3 grid (every k0 resolved there, k0 h <
    0.625): the nested iteration's finest level needs within two V-cycles of
    the counts Table 3 prints, and fewer than the V-cycles from zero for the
    smaller k0 (tests/golden/table3_fmg_gmres3.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_fmg_gmres3.txt")
    gold = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, pts, cyc = line.split()[:3]
            gold[(float(k), int(pts))] = int(cyc)
    for k in (0.25, 0.5, 1.0, 2.0, 4.0):
        c = W.paper_gmres(dim=3, k=k, n=257)
        c["opts"]["precision"] = "fp64"
        plan = csff.Plan(c["problem"], c["opts"])
        u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
        st, info, cyc = plan.solve_fmg(c["eta"], u)
        assert st == csff.OK and info[0]["rel_res"] <= 1e-6
        assert abs(cyc[0][-1] - gold[(k, 256)]) <= 2, (k, cyc[0], gold[(k, 256)])
        if k <= 0.5:
            u0 = torch.zeros_like(u)
            _, inf0 = plan.solve(c["eta"], u0)
            assert cyc[0][-1] < inf0[0]["cycles"]
        plan.close()
