"""CUDA path (through the C ABI) against the CPU FP64 oracle on the same
seeded inputs.  Tolerances: FP64 kernels agree to rounding (1e-12 of the
magnitude of the terms summed); FP32 kernels to 1e-5 of it (a few FP32 ulps
over the ~12 terms of a stencil update); far-field maps to 1e-6 relative L2 in
FP64 (the stated FP64 target; measured far below it) and 1e-5 after mixed
refinement, over the angles whose condition number kappa keeps the FP64
rounding floor under a tenth of the tolerance."""
import math

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


def cases():
    c2 = W.small_2d(n=33)
    c3 = {"name": "3d-n17", "problem": W.problem(3, 17, 6.0, math.pi / 6, 1.5, [W.gauss(-0.7, 2.0, (0.4, -0.3, 0.2))]),
          "opts": {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5, "rel_tol": 1e-10,
                   "max_cycles": 100},
          "eta": np.array([[0.6, 0.0, 0.8]]), "alphas": W.angle_set_3d(8, 4)}
    c2b = W.small_2d(n=65)
    c2b["problem"]["gaussians"] = [W.gauss(-0.3 - 0.05j, 2.0, (0.5, -0.3, 0.0)), W.gauss(-0.2, 1.0, (-0.5, 0.5, 0.0))]
    c2b["name"] = "2d-n65-two-gaussians"
    # red-black V(1,1) in 2D runs the fused kernels (levels >= 33^2 in one CTA)
    c2r = W.mixed_2d(5.0, n=129)
    c2r["problem"]["hi"], c2r["problem"]["lo"] = 12.0, -12.0
    c2r["opts"].update(coarsest_n=5, rel_tol=1e-10)
    c2r["name"] = "2d-n129-rbgs-fused"
    c2s = dict(c2r, name="2d-n65-rbgs-fused", problem=dict(c2r["problem"], n=65))
    return [c2, c2b, c3, c2r, c2s]


CASES = cases()
IDS = [c["name"] for c in CASES]
TOL = {np.complex128: 1e-12, np.complex64: 1e-5}


def _tol(dt):
    return TOL[np.complex128] if dt == torch.complex128 else TOL[np.complex64]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def setup(request, csff):
    c = CASES[request.param]
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    levels = O.make_hierarchy(p, c["opts"]["coarsest_n"])
    yield c, plan, p, levels
    plan.close()


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64], ids=["fp64", "fp32"])
def test_residual(setup, dt):
    c, plan, p, levels = setup
    for l in (0, len(levels) - 2):
        lv = levels[l]
        shp = (lv.m,) * p.dim
        u = W.rand_complex(shp, 100 + l)
        b = W.rand_complex(shp, 200 + l, scale=50.0)
        if dt == torch.complex64:
            u = u.astype(np.complex64).astype(np.complex128)
            b = b.astype(np.complex64).astype(np.complex128)
        r = torch.empty(lv.m ** p.dim, dtype=dt, device="cuda")
        plan.residual(l, dev(u, dt), dev(b, dt), r)
        ref = O.residual(lv, u, b)
        scale = np.abs(b).max() + (abs(lv.c) * 4 * p.dim + np.abs(lv.q).max()) * np.abs(u).max()
        assert np.abs(host(r, shp) - ref).max() <= _tol(dt) * scale


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64], ids=["fp64", "fp32"])
@pytest.mark.parametrize("smoother", ["jacobi", "rbgs"])
def test_smoother(setup, csff, dt, smoother):
    c, _, p, levels = setup
    opts = dict(c["opts"], smoother=smoother, omega=0.6)
    plan = csff.Plan(c["problem"], opts)
    oo = O.opts_from_dict(opts)
    l = 0
    lv = levels[l]
    shp = (lv.m,) * p.dim
    u0 = W.rand_complex(shp, 300)
    b = W.rand_complex(shp, 301, scale=50.0)
    if dt == torch.complex64:
        u0 = u0.astype(np.complex64).astype(np.complex128)
        b = b.astype(np.complex64).astype(np.complex128)
    ut = dev(u0, dt)
    plan.smooth(l, ut, dev(b, dt), sweeps=3)
    ref = u0
    for _ in range(3):
        ref = O._smooth(lv, ref, b, oo)
    scale = np.abs(ref).max() + np.abs(u0).max()
    assert np.abs(host(ut, shp) - ref).max() <= 10 * _tol(dt) * scale
    plan.close()


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64], ids=["fp64", "fp32"])
def test_restrict_and_prolong(setup, dt):
    c, plan, p, levels = setup
    for l in range(len(levels) - 1):
        f, cl = levels[l], levels[l + 1]
        r = W.rand_complex((f.m,) * p.dim, 400 + l)
        e = W.rand_complex((cl.m,) * p.dim, 500 + l)
        uf = W.rand_complex((f.m,) * p.dim, 600 + l)
        if dt == torch.complex64:
            r, e, uf = (x.astype(np.complex64).astype(np.complex128) for x in (r, e, uf))
        bc = torch.empty(cl.m ** p.dim, dtype=dt, device="cuda")
        plan.restrict(l, dev(r, dt), bc)
        assert np.abs(host(bc, (cl.m,) * p.dim) - O.restrict_fw(r)).max() <= _tol(dt) * np.abs(r).max() * 2
        ut = dev(uf, dt)
        plan.prolong_add(l, dev(e, dt), ut)
        ref = uf + O.prolong(e)
        assert np.abs(host(ut, (f.m,) * p.dim) - ref).max() <= _tol(dt) * (np.abs(uf).max() + np.abs(e).max()) * 2


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64], ids=["fp64", "fp32"])
def test_coarse_solve(setup, dt):
    c, plan, p, levels = setup
    lv = levels[-1]
    shp = (lv.m,) * p.dim
    b = W.rand_complex(shp, 700)
    if dt == torch.complex64:
        b = b.astype(np.complex64).astype(np.complex128)
    u = torch.empty(lv.m ** p.dim, dtype=dt, device="cuda")
    plan.coarse_solve(dev(b, dt), u)
    ref = O.coarse_solve(O.coarse_factor(lv), b)
    tol = 1e-11 if dt == torch.complex128 else 1e-5
    assert np.abs(host(u, shp) - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64], ids=["fp64", "fp32"])
def test_norm(setup, dt):
    c, plan, p, levels = setup
    v = W.rand_complex((levels[0].m,) * p.dim, 800, scale=3.0)
    if dt == torch.complex64:
        v = v.astype(np.complex64).astype(np.complex128)
    got = plan.norm2(0, dev(v, dt))
    assert abs(got - O.norm2(v)) <= 1e-13 * O.norm2(v)


def test_vcycle_fp64(setup):
    c, plan, p, levels = setup
    oo = O.opts_from_dict(c["opts"])
    lu = O.coarse_factor(levels[-1])
    shp = (levels[0].m,) * p.dim
    u0 = W.rand_complex(shp, 900)
    b = W.rand_complex(shp, 901, scale=20.0)
    ut = dev(u0)
    plan.vcycle(ut, dev(b))
    ref = O.vcycle(levels, lu, 0, u0, b, oo)
    assert np.abs(host(ut, shp) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_vcycle_fp32(setup):
    """FP32 V-cycle against the FP64 oracle cycle from the same FP32-rounded inputs."""
    c, plan, p, levels = setup
    oo = O.opts_from_dict(c["opts"])
    lu = O.coarse_factor(levels[-1])
    shp = (levels[0].m,) * p.dim
    u0 = W.rand_complex(shp, 902).astype(np.complex64).astype(np.complex128)
    b = W.rand_complex(shp, 903, scale=20.0).astype(np.complex64).astype(np.complex128)
    ut = dev(u0, torch.complex64)
    plan.vcycle(ut, dev(b, torch.complex64))
    ref = O.vcycle(levels, lu, 0, u0, b, oo)
    assert np.abs(host(ut, shp) - ref).max() <= 1e-4 * np.abs(ref).max()


def test_vcycles_with_the_rhs_changed_in_between(setup):
    """Three FP32 V-cycles in a row on the plan's stream, the right-hand side
    doubled in place by a torch kernel on that stream just before each (the
    fused up tiles copy their fine windows before they wait for the kernel
    before them): each cycle against the oracle's cycle from the GPU's
    previous iterate and the doubled right-hand side."""
    c, plan, p, levels = setup
    oo = O.opts_from_dict(c["opts"])
    lu = O.coarse_factor(levels[-1])
    shp = (levels[0].m,) * p.dim
    u0 = W.rand_complex(shp, 904).astype(np.complex64).astype(np.complex128)
    b = W.rand_complex(shp, 905, scale=20.0).astype(np.complex64).astype(np.complex128)
    ut = dev(u0, torch.complex64)
    bt = dev(b, torch.complex64)
    prev = u0
    for _ in range(3):
        bt.mul_(2.0)
        b = 2.0 * b
        plan.vcycle(ut, bt)
        ref = O.vcycle(levels, lu, 0, prev, b, oo)
        got = host(ut, shp).astype(np.complex128)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
        prev = got


def test_solve_fp64_history_and_far_field(setup):
    """Per-cycle residual history, cycle count, solution and far-field map."""
    c, plan, p, levels = setup
    eta = c["eta"]
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(eta, u)
    res = O.mg_solve(p, O.rhs(p, eta[0]), O.opts_from_dict(c["opts"]))
    assert info[0]["cycles"] == res.cycles
    h_gpu, h_or = np.array(info[0]["history"]), np.array(res.history)
    # the relative residual carries a rounding floor of ~eps ||A|| ||u|| / ||b|| ~ 1e-15
    assert np.allclose(h_gpu, h_or, rtol=1e-6, atol=1e-15)
    ug = host(u, res.u.shape)
    assert np.linalg.norm(ug - res.u) <= 1e-9 * np.linalg.norm(res.u)
    al = c["alphas"]
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    plan.far_field(eta, u, al, F)
    Fo = O.far_field_value(*O.far_field(p, res.u, eta[0], al))
    assert np.linalg.norm(F.cpu().numpy() - Fo) <= 1e-6 * np.linalg.norm(Fo)
    # far field from the same solution: rounding-level agreement
    Fs = O.far_field_value(*O.far_field(p, ug, eta[0], al))
    assert np.linalg.norm(F.cpu().numpy() - Fs) <= 1e-12 * np.linalg.norm(Fs)


@pytest.mark.parametrize("lo,hi", [(-10.0, 10.0), (-9.0, 11.0)], ids=["symmetric-box", "shifted-box"])
def test_far_field_on_symmetric_and_shifted_boxes(csff, lo, hi):
    """Far field on a box symmetric about 0 and on a shifted one against the
    oracle on the same solution, with outgoing directions that include
    unpaired x-components."""
    c = W.small_2d(n=65)
    c["problem"]["lo"], c["problem"]["hi"] = lo, hi
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    plan.solve(c["eta"], u)
    ug = host(u, (p.m,) * 2)
    al = np.vstack([c["alphas"][::7], W.angle_set_2d(13)])
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    plan.far_field(c["eta"], u, al, F)
    m, e2, tn = O.far_field(p, ug, c["eta"][0], al, return_terms_norm=True)
    Fo = O.far_field_value(m, e2)
    assert np.abs(F.cpu().numpy() - Fo).max() <= 1e-13 * (tn * 2.0 ** e2).max()


def test_rhs_with_factor_overflow(csff):
    """45-degree incidence, k = 52, w = 1 on [-20,20]^2: the incident wave alone
    exceeds the FP64 range at the upstream corner, chi u_in does not; the
    device source matches the oracle's."""
    c = W.mixed_2d(52.0, n=65)
    c["problem"]["gaussians"] = [W.gauss(-1.0, 1.0)]
    c["opts"]["coarsest_n"] = 5
    plan = csff.Plan(c["problem"], c["opts"])
    eta = np.array([[math.sqrt(0.5), math.sqrt(0.5)]])
    b = torch.empty(plan.N, dtype=torch.complex128, device="cuda")
    plan.rhs(eta, b)
    ref = O.rhs(O.problem_from_dict(c["problem"]), eta[0]).ravel()
    got = b.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_rhs(setup):
    c, plan, p, levels = setup
    eta = np.vstack([c["eta"], -c["eta"]])
    b = torch.empty(2 * plan.N, dtype=torch.complex128, device="cuda")
    plan.rhs(eta, b)
    for r in range(2):
        ref = O.rhs(p, eta[r]).ravel()
        got = b[r * plan.N:(r + 1) * plan.N].cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_chi_zero_gives_exact_zero(csff):
    c = W.small_2d(n=33)
    c["problem"]["gaussians"] = [W.gauss(0.0, 2.0)]
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.full((plan.N,), 1.0 + 1.0j, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(c["eta"], u)
    assert st == csff.OK and torch.count_nonzero(u).item() == 0
    F = torch.ones(len(c["alphas"]), dtype=torch.complex128, device="cuda")
    plan.far_field(c["eta"], u, c["alphas"], F)
    assert torch.count_nonzero(F).item() == 0


def test_empty_calls(csff):
    c = W.small_2d(n=33)
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    F = torch.zeros(1, dtype=torch.complex128, device="cuda")
    assert plan.far_field(np.zeros((0, 2)), u, c["alphas"][:1], F) == csff.OK
    assert plan.far_field(c["eta"], u, np.zeros((0, 2)), F) == csff.OK


def test_nonfinite_input_is_reported(csff):
    c = W.small_2d(n=33)
    c["problem"]["gaussians"] = [W.gauss(float("nan"), 2.0)]
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(c["eta"], u, ok=(csff.ERR_NONFINITE,))
    assert st == csff.ERR_NONFINITE and info[0]["status"] == csff.ERR_NONFINITE


def test_divergence_is_detected_like_the_oracle(csff):
    """An amplifying medium (Im chi > 0) makes the V-cycle iteration grow; the
    library stops with DIVERGED where the oracle's residual history grows too."""
    c = W.small_2d(n=65)
    c["problem"]["gaussians"] = [W.gauss(-0.5 + 0.1j, 2.0, (0.7, -0.4, 0.0)), W.gauss(-0.2, 1.0, (-1.0, 2.0, 0.0))]
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(c["eta"], u, ok=(csff.ERR_DIVERGED,))
    p = O.problem_from_dict(c["problem"])
    oo = O.opts_from_dict(c["opts"])
    oo.max_cycles = info[0]["cycles"]
    res = O.mg_solve(p, O.rhs(p, c["eta"][0]), oo)
    assert st == csff.ERR_DIVERGED
    assert np.allclose(info[0]["history"], res.history, rtol=1e-6)
    h = res.history
    assert h[-1] > h[-2] > h[-3] > h[-4]


def _cone_rel_err(Fg, Fo, tn, e2, eps_work, tol):
    """rel-L2 over the angles with kappa * eps_work <= tol / 10 (kappa from the oracle)."""
    F_o = O.far_field_value(Fo, e2)
    kappa = tn / np.maximum(np.abs(Fo), 1e-300)
    cone = kappa * eps_work <= tol / 10
    return cone, np.linalg.norm(Fg[cone] - F_o[cone]) / np.linalg.norm(F_o[cone])


@pytest.mark.parametrize("refine_fp64", [0, 1])
@pytest.mark.parametrize("k,n", [(5.0, 129), (10.0, 257)])
def test_mixed_refinement_solution_and_far_field(csff, k, n, refine_fp64):
    """FP32 V-cycles inside the refinement, its residual and update in
    double-float (default) or in FP64 (refine_fp64)."""
    c = W.mixed_2d(k, n=n)
    c["opts"]["coarsest_n"] = 9
    c["opts"]["precision"] = "mixed"
    c["opts"]["refine_fp64"] = refine_fp64
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    eta = c["eta"]
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(eta, u)
    assert st == csff.OK and info[0]["rel_res"] <= 1e-8
    ug = host(u, (p.m,) * 2)
    b = O.rhs(p, eta[0])
    lv = O.make_level(p, p.n)
    assert O.norm2(O.residual(lv, ug, b)) <= 1.01e-8 * O.norm2(b)
    res = O.mg_solve(p, b, O.opts_from_dict(c["opts"]))
    al = c["alphas"]
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    plan.far_field(eta, u, al, F)
    m, e2, tn = O.far_field(p, res.u, eta[0], al, return_terms_norm=True)
    cone, err = _cone_rel_err(F.cpu().numpy(), m, tn, e2, 1e-8, 1e-5)
    assert cone.sum() >= 3 and err <= 1e-5


@pytest.mark.parametrize("refine_fp64", [0, 1])
@pytest.mark.parametrize("dim,n", [(2, 257), (3, 65)])
def test_mixed_refinement_reaches_tight_tolerances(csff, dim, n, refine_fp64):
    """The refinement's residual and update carry pairs of FP32 words (about 48
    significant bits; exact products for the 2D and 3D centre weights 4 and 6),
    or FP64 words with refine_fp64, so a mixed solve asked for 1e-11 meets it
    under the oracle's FP64 operator."""
    c = W.mixed_2d(10.0, n=n) if dim == 2 else W.big_3d(n=n, n_rhs=1)
    c["opts"].update(precision="mixed", rel_tol=1e-11, max_cycles=400, refine_fp64=refine_fp64)
    if dim == 2:
        c["opts"]["coarsest_n"] = 9
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    eta = c["eta"]
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve(eta[:1], u)
    assert st == csff.OK and info[0]["rel_res"] <= 1e-11
    ug = host(u, (p.m,) * dim)
    b = O.rhs(p, eta[0])
    lv = O.make_level(p, p.n)
    assert O.norm2(O.residual(lv, ug, b)) <= 1.05e-11 * O.norm2(b)
    plan.close()


@pytest.mark.parametrize("k", [20.0, 40.0])
def test_adaptive_refinement_meets_the_tolerance_in_fewer_cycles(csff, k):
    """adaptive_inner sizes each refinement step from the previous step's
    per-cycle reduction factor: the solve meets the same tolerance (re-checked
    with the oracle's FP64 operator) in at most the cycles of the fixed
    schedule, and a solve from a converged guess stops after one step."""
    c = W.mixed_2d(k, n=513)
    c["opts"].update(precision="mixed", inner_cycles=6, coarsest_n=9)
    p = O.problem_from_dict(c["problem"])
    eta = c["eta"][:1]
    runs = {}
    for adaptive in (0, 1):
        plan = csff.Plan(c["problem"], dict(c["opts"], adaptive_inner=adaptive))
        u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
        st, info = plan.solve(eta, u)
        assert st == csff.OK and info[0]["rel_res"] <= 1e-8
        runs[adaptive] = (plan, u, info[0])
    assert runs[1][2]["cycles"] <= runs[0][2]["cycles"]
    ug = host(runs[1][1], (p.m,) * 2)
    b = O.rhs(p, eta[0])
    lv = O.make_level(p, p.n)
    assert O.norm2(O.residual(lv, ug, b)) <= 1.01e-8 * O.norm2(b)
    plan, u, _ = runs[1]
    st, info = plan.solve(eta, u, use_guess=True)
    assert st == csff.OK and info[0]["refinements"] == 1
    for pl, _, _ in runs.values():
        pl.close()


def test_fp64_far_field_matches_on_paper_window_variant(csff):
    """Same grid, k and smoother as the 1025^2 case at n=257, with w = 28/k^2
    (largest term below e^14): FP64 maps agree to the 1e-6 target over all
    angles."""
    c = W.paper_window(W.mixed_2d(10.0, n=257))
    c["opts"]["coarsest_n"] = 9
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    plan.solve(c["eta"], u)
    res = O.mg_solve(p, O.rhs(p, c["eta"][0]), O.opts_from_dict(c["opts"]))
    al = c["alphas"]
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    plan.far_field(c["eta"], u, al, F)
    Fo = O.far_field_value(*O.far_field(p, res.u, c["eta"][0], al))
    assert np.linalg.norm(F.cpu().numpy() - Fo) <= 1e-6 * np.linalg.norm(Fo)


def test_far_field_extended_range_k40(csff):
    """k = 40 on [-20,20]^2: terms beyond the FP64 range.  With exponent output
    the map stays finite and matches the oracle's mantissa/exponent pairs
    within the backward-error bound (eps * sum|terms| per angle)."""
    c = W.mixed_2d(40.0, n=257)
    c["opts"]["coarsest_n"] = 9
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    u0 = np.zeros((p.m,) * 2, complex)
    al = c["alphas"][::20]
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    Fe = torch.zeros(len(al), dtype=torch.int32, device="cuda")
    plan.far_field(c["eta"], dev(u0), al, F, Fe)
    m, e2, tn = O.far_field(p, u0, c["eta"][0], al, return_terms_norm=True)
    Fg, eg = F.cpu().numpy(), Fe.cpu().numpy().astype(np.int64)
    assert np.all(np.isfinite(Fg)) and eg.max() > 0
    for a in range(len(al)):
        d = Fg[a] * 2.0 ** float(eg[a] - e2[a]) - m[a]
        assert abs(d) <= 1e-12 * tn[a] + 1e-300


def test_far_field_skips_negligible_blocks_within_the_bound(csff):
    """k = 20 on [-20,20]^2 (257^2): most stage-1 blocks carry terms far below
    the largest ones along the rotated contour and are skipped; the map still
    meets the per-angle bound 1e-13 * sum_j |term_j| against the oracle."""
    c = W.mixed_2d(20.0, n=257)
    c["opts"].update(coarsest_n=9, rel_tol=1e-8)
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    plan.solve(c["eta"], u)
    al = c["alphas"]
    F = torch.zeros(len(al), dtype=torch.complex128, device="cuda")
    E = torch.zeros(len(al), dtype=torch.int32, device="cuda")
    plan.far_field(c["eta"], u, al, F, E)
    work = plan.far_field_work()
    assert 0.0 < work < 0.8
    got = F.cpu().numpy() * 2.0 ** E.cpu().numpy().astype(np.float64)
    mant, e2, tn = O.far_field(p, host(u, (p.m,) * 2), c["eta"][0], al, return_terms_norm=True)
    ref = O.far_field_value(mant, e2)
    assert np.all(np.abs(got - ref) <= 1e-13 * tn * 2.0 ** e2)
    plan.close()
