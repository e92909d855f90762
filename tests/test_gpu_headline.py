"""Parity on the 1025^2 workload itself (box [-20,20]^2, rotation pi/6,
chi = -exp(-|x|^2/4), RB-GS V(1,1), 8 levels, 9^2 coarsest grid): the kernels
that run only at this size -- the fused tiles of 16 coarse points on the
1025^2 and 513^2 levels, in FP32 and in FP64 -- against the oracle's V-cycle element by
element, full mixed solves re-checked with the oracle's FP64 operator, their
far fields against the oracle's sum on the same solution, and the batched
kernel with 1025^2 instances on 16-point tiles.  GPU only."""
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


def host(t, shape):
    return t.cpu().numpy().astype(np.complex128).reshape(shape)


@pytest.fixture(scope="module", params=[5.0, 40.0], ids=["k5", "k40"])
def headline(request):
    c = W.mixed_2d(request.param)
    p = O.problem_from_dict(c["problem"])
    levels = O.make_hierarchy(p, c["opts"]["coarsest_n"])
    assert [lv.n for lv in levels] == [1025, 513, 257, 129, 65, 33, 17, 9]
    return c, p, levels, O.coarse_factor(levels[-1])


@pytest.mark.parametrize("refine_fp64", [0, 1], ids=["df", "fp64"])
def test_fp32_vcycle_at_1025_matches_oracle(csff, headline, refine_fp64):
    """One FP32 V-cycle through the 16-point tiles of the 1025^2 and 513^2
    levels (and the 8-point tiles and coarse-level block below), against the FP64 oracle cycle
    from the same FP32-rounded inputs.  With refine_fp64 the coarsest solve
    runs in FP64."""
    c, p, levels, lu = headline
    plan = csff.Plan(c["problem"], dict(c["opts"], precision="mixed", refine_fp64=refine_fp64))
    shp = (p.m, p.m)
    u0 = W.rand_complex(shp, 1902).astype(np.complex64).astype(np.complex128)
    b = W.rand_complex(shp, 1903, scale=20.0).astype(np.complex64).astype(np.complex128)
    ut = dev(u0, torch.complex64)
    plan.vcycle(ut, dev(b, torch.complex64))
    ref = O.vcycle(levels, lu, 0, u0, b, O.opts_from_dict(c["opts"]))
    assert np.abs(host(ut, shp) - ref).max() <= 1e-4 * np.abs(ref).max()
    plan.close()


def test_fp64_vcycle_at_1025_matches_oracle(csff, headline):
    """One FP64 V-cycle (FP64 16-point tiles on the 1025^2 and 513^2 levels)
    against the oracle cycle."""
    c, p, levels, lu = headline
    plan = csff.Plan(c["problem"], dict(c["opts"], precision="fp64"))
    shp = (p.m, p.m)
    u0 = W.rand_complex(shp, 1904)
    b = W.rand_complex(shp, 1905, scale=20.0)
    ut = dev(u0)
    plan.vcycle(ut, dev(b))
    ref = O.vcycle(levels, lu, 0, u0, b, O.opts_from_dict(c["opts"]))
    assert np.abs(host(ut, shp) - ref).max() <= 1e-11 * np.abs(ref).max()
    plan.close()


@pytest.mark.parametrize("refine_fp64", [1, 0], ids=["fp64", "df"])
def test_mixed_solve_and_far_field_at_1025(csff, headline, refine_fp64):
    """The bench's solve (FP32 cycles inside the refinement, adaptive schedule
    of at most six cycles a step): its solution meets 1e-8 under the oracle's
    FP64 operator, and its far field at every 20th of the 720 angles meets the
    backward-error bound 1e-12 sum_j |term_j| against the oracle's sum on the
    same solution (mantissa and exponent per angle: at k = 40 the terms leave
    the FP64 range)."""
    c, p, levels, lu = headline
    opts = dict(c["opts"], precision="mixed", inner_cycles=6, adaptive_inner=1, refine_fp64=refine_fp64)
    plan = csff.Plan(c["problem"], opts)
    eta = c["eta"]
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(eta, u)
    assert st == csff.OK and info[0]["rel_res"] <= 1e-8
    ug = host(u, (p.m, p.m))
    b = O.rhs(p, eta[0])
    assert O.norm2(O.residual(levels[0], ug, b)) <= 1.01e-8 * O.norm2(b)
    al = c["alphas"][::20]
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    E = torch.zeros(len(al), dtype=torch.int32, device="cuda")
    plan.far_field(eta, u, al, F, E)
    mant, e2, tn = O.far_field(p, ug, eta[0], al, return_terms_norm=True)
    Fg, eg = F.cpu().numpy(), E.cpu().numpy().astype(np.int64)
    for a in range(len(al)):
        d = Fg[a] * 2.0 ** float(eg[a] - e2[a]) - mant[a]
        assert abs(d) <= 1e-12 * tn[a], (a, abs(d), tn[a])
    plan.close()


def test_batch_with_1025_instances_on_16_point_tiles(csff):
    """Uneven batch whose largest instances are 1025^2, with 16-point tiles
    fixed on the large levels: every instance meets 1e-8 under the oracle's
    operator and runs the single-plan iteration (same cycles and history)."""
    cs = W.batch_2d(5, seed=77, sizes=(257, 513, 1025))
    assert any(c["problem"]["n"] == 1025 for c in cs)
    for c in cs:
        c["opts"].update(precision="mixed", inner_cycles=3, refine_fp64=1)
    b = csff.Batch([c["problem"] for c in cs], cs[0]["opts"])
    b.set_tiles(16)
    eta = np.vstack([c["eta"] for c in cs])
    st, infos = b.solve(eta)
    assert st == csff.OK
    for i, c in enumerate(cs):
        p = O.problem_from_dict(c["problem"])
        rhs = O.rhs(p, c["eta"][0])
        u = b.solution(i).cpu().numpy().reshape((p.m, p.m))
        lv = O.make_level(p, p.n)
        assert O.norm2(O.residual(lv, u, rhs)) <= 1.01e-8 * O.norm2(rhs)
        plan = csff.Plan(c["problem"], c["opts"])
        us = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
        _, inf1 = plan.solve(c["eta"], us)
        assert inf1[0]["cycles"] == infos[i]["cycles"]
        assert np.allclose(inf1[0]["history"], infos[i]["history"], rtol=1e-5, atol=1e-14)
        plan.close()
    b.close()
