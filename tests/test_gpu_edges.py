"""Edge cases through the C ABI against the oracle: a hierarchy of one level
(the coarsest grid is the whole problem), the largest grid the bench runs
(4097^2, FP32 arrays beyond the L2 cache), batches of one instance and with an
instance whose source vanishes.  GPU only."""
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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a).ravel()).to("cuda")
    return t.to(dtype) if dtype is not None else t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_level_plan_is_the_direct_solve(csff, precision):
    """n = coarsest_n = 5: the V-cycle is the coarsest solve itself, so one
    cycle (FP64) or one refinement step (mixed) reaches the direct solution;
    full multigrid has no level to iterate on and returns it too."""
    c = W.small_2d(n=5)
    c["opts"].update(coarsest_n=5, precision=precision, rel_tol=1e-10)
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(c["eta"], u)
    assert st == csff.OK and info[0]["rel_res"] <= 1e-10
    ref = O.direct_solve(p, O.rhs(p, c["eta"][0]))
    got = u.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    if precision == "fp64":
        assert info[0]["cycles"] == 1
        uf = torch.zeros_like(u)
        st, _, cyc = plan.solve_fmg(c["eta"], uf)
        assert st == csff.OK and cyc == [[]]
        assert np.abs(uf.cpu().numpy().reshape(ref.shape) - ref).max() <= 1e-12 * np.abs(ref).max()
    plan.close()


def test_fp32_vcycle_on_the_largest_grid(csff):
    """4097^2 (134 MB per FP32 array, beyond the L2 cache; 16-point tiles on
    the 4097^2 to 513^2 levels): one FP32 V-cycle against the
    oracle's cycle from the same FP32-rounded inputs, element by element."""
    c = W.mixed_2d(40.0, n=4097)
    c["opts"].update(coarsest_n=9, precision="mixed")
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    levels = O.make_hierarchy(p, 9)
    shp = (p.m, p.m)
    u0 = W.rand_complex(shp, 4097).astype(np.complex64).astype(np.complex128)
    b = W.rand_complex(shp, 4098, scale=20.0).astype(np.complex64).astype(np.complex128)
    ut = dev(u0, torch.complex64)
    plan.vcycle(ut, dev(b, torch.complex64))
    ref = O.vcycle(levels, O.coarse_factor(levels[-1]), 0, u0, b, O.opts_from_dict(c["opts"]))
    got = ut.cpu().numpy().astype(np.complex128).reshape(shp)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    plan.close()


def test_vcycles_on_the_headline_grid_with_the_rhs_changed_in_between(csff):
    """1025^2 (16-point tiles on the 1025^2 and 513^2 levels): three FP32 V-cycles in a
    row on the plan's stream with the right-hand side doubled in place by a
    torch kernel before each, every cycle against the oracle's from the GPU's
    previous iterate."""
    c = W.mixed_2d(20.0)
    c["opts"]["precision"] = "mixed"
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    levels = O.make_hierarchy(p, c["opts"]["coarsest_n"])
    lu = O.coarse_factor(levels[-1])
    oo = O.opts_from_dict(c["opts"])
    shp = (p.m, p.m)
    prev = W.rand_complex(shp, 906).astype(np.complex64).astype(np.complex128)
    b = W.rand_complex(shp, 907, scale=20.0).astype(np.complex64).astype(np.complex128)
    ut = dev(prev, torch.complex64)
    bt = dev(b, torch.complex64)
    for _ in range(3):
        bt.mul_(2.0)
        b = 2.0 * b
        plan.vcycle(ut, bt)
        ref = O.vcycle(levels, lu, 0, prev, b, oo)
        got = ut.cpu().numpy().astype(np.complex128).reshape(shp)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
        prev = got
    plan.close()


def test_batch_of_one_and_with_a_vanishing_source(csff):
    """A batch of one instance runs the single-plan iteration; in a batch whose
    second instance has chi = 0 (so b = 0) that instance ends at once with
    u = 0 while the others converge."""
    cs = W.batch_2d(3, seed=5, sizes=(65, 129))
    for c in cs:
        c["opts"].update(precision="mixed", inner_cycles=3, refine_fp64=1)
    one = csff.Batch([cs[0]["problem"]], cs[0]["opts"])
    st, inf = one.solve(cs[0]["eta"])
    assert st == csff.OK and inf[0]["rel_res"] <= 1e-8
    plan = csff.Plan(cs[0]["problem"], cs[0]["opts"])
    us = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    _, inf1 = plan.solve(cs[0]["eta"], us)
    assert inf1[0]["cycles"] == inf[0]["cycles"]
    plan.close()
    one.close()
    cs[1]["problem"]["gaussians"] = [W.gauss(0.0, 2.0)]
    b = csff.Batch([c["problem"] for c in cs], cs[0]["opts"])
    eta = np.vstack([c["eta"] for c in cs])
    st, infos = b.solve(eta)
    assert st == csff.OK
    assert infos[1]["cycles"] == 0 and torch.count_nonzero(b.solution(1)).item() == 0
    for i in (0, 2):
        p = O.problem_from_dict(cs[i]["problem"])
        rhs = O.rhs(p, cs[i]["eta"][0])
        u = b.solution(i).cpu().numpy().reshape((p.m, p.m))
        assert O.norm2(O.residual(O.make_level(p, p.n), u, rhs)) <= 1.01e-8 * O.norm2(rhs)
    b.close()
