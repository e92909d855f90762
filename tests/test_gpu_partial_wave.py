"""The partial-wave path (Sec. 5.2-5.3) through the C-ABI against the oracle:
user potential + user right-hand side solves (V(1,1)/GMRES(3) on the
contour, FP64 and mixed precision), the 1D contour functions, the separable
integrals, and the cross sections end to end."""
import math

import numpy as np
import pytest

import oracle.partial_wave as PW
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4461_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128).ravel()).to("cuda")


def _plan(csff, c):
    plan = csff.Plan(c["problem"], c["opts"])
    plan.set_schroedinger(c["E"], dev(c["V"]))
    return plan


@pytest.mark.parametrize("E", [-1.5, 1.0, 2.5])
def test_solve_with_user_potential_matches_direct_solve(csff, E):
    c = W.partial_wave(E, n=129)
    plan = _plan(csff, c)
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve_schroedinger(dev(c["f"]), u)
    assert st == csff.OK and info["rel_res"] <= 1e-10
    ref = PW.solve(E, 129)
    got = u.cpu().numpy().reshape(ref.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    plan.close()


def test_sampled_coefficients_through_set_potential(csff):
    """The same problem given as coefficient samples (the oracle's q = 2E - 2V
    and 2 phi) through csff_plan_set_potential / csff_solve_rhs: the solution
    matches the direct solve and the device-formed path."""
    E, n = 1.0, 129
    c = W.partial_wave(E, n=n)
    _, _, ph = PW.fields(n)
    plan = csff.Plan(c["problem"], c["opts"])
    plan.set_potential(dev(PW.q_of(E, n)))
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve_rhs(dev(2.0 * ph), u)
    assert st == csff.OK and info["rel_res"] <= 1e-10
    ref = PW.solve(E, n)
    got = u.cpu().numpy().reshape(ref.shape)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    plan2 = _plan(csff, c)
    u2 = torch.zeros(plan2.N, dtype=torch.complex128, device="cuda")
    st2, info2 = plan2.solve_schroedinger(dev(c["f"]), u2)
    assert st2 == csff.OK and info2["cycles"] == info["cycles"]
    assert np.linalg.norm(u2.cpu().numpy().reshape(ref.shape) - got) <= 1e-12 * np.linalg.norm(got)
    plan.close()
    plan2.close()


def test_mixed_precision_solve_with_user_potential(csff):
    c = W.partial_wave(2.0, n=257)
    c["opts"].update(precision="mixed", inner_cycles=2, rel_tol=1e-9)
    plan = _plan(csff, c)
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve_schroedinger(dev(c["f"]), u)
    assert st == csff.OK and info["rel_res"] <= 1e-9
    ref = PW.solve(2.0, 257)
    got = u.cpu().numpy().reshape(ref.shape)
    assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)
    plan.close()


def test_vcycle_history_matches_oracle(csff):
    import oracle.csff_oracle as O
    c = W.partial_wave(1.5, n=129)
    plan = _plan(csff, c)
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, info = plan.solve_schroedinger(dev(c["f"]), u)
    o = O.MGOptions(smoother="gmres", nu1=1, nu2=1, coarsest_n=5, rel_tol=1e-10, max_cycles=200, krylov_m=3)
    r = PW.mg_solve(1.5, 129, o)
    assert info["cycles"] == r.cycles
    np.testing.assert_allclose(info["history"], r.history, rtol=1e-6, atol=1e-15)
    plan.close()


@pytest.mark.parametrize("gamma_deg", [0.0, 8.5])
def test_contour_functions_match_oracle(csff, gamma_deg):
    n = 257
    g = math.radians(gamma_deg)
    c = W.partial_wave(1.0, n=n, gamma=g)
    lam, phi = csff.contour_bound_state(c["v1"], c["h"], g, -1.0)
    lo, po = PW.bound_states(n, gamma=g)[0]
    assert abs(lam - lo) <= 1e-10
    assert np.abs(phi - po).max() <= 1e-9 * np.abs(po).max()
    for k in (0.3, 1.4, 2.6):
        rs = csff.contour_regular_solution(c["v1"], c["h"], g, k)
        ro = PW.regular_solution(k, n, gamma=g)
        assert np.abs(rs - ro).max() <= 1e-9 * np.abs(ro).max(), k


def test_separable_sum_matches_oracle(csff):
    n = 129
    c = W.partial_wave(1.0, n=n)
    plan = _plan(csff, c)
    m = n - 2
    X = W.rand_complex((7, m), 61)
    Y = W.rand_complex((7, m), 62)
    u = W.rand_complex((m, m), 63)
    out = plan.separable_sum(dev(X).reshape(7, m), dev(Y).reshape(7, m), dev(c["f"]), dev(c["w"]), dev(u))
    ref = PW.contract(X, Y, c["f"] - c["w"] * u, n)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    out2 = plan.separable_sum(dev(X).reshape(7, m), dev(Y).reshape(7, m), dev(c["f"]))
    ref2 = PW.contract(X, Y, c["f"], n)
    assert np.abs(out2.cpu().numpy() - ref2).max() <= 1e-12 * np.abs(ref2).max()
    plan.close()


def test_cross_sections_end_to_end(csff):
    # solve on the GPU, 1D functions from the library, integrals on the GPU;
    # against the oracle's amplitudes on the same grid
    E, n = 1.0785, 257
    c = W.partial_wave(E, n=n)
    plan = _plan(csff, c)
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    st, _ = plan.solve_schroedinger(dev(c["f"]), u)
    assert st == csff.OK
    g = c["gamma"]
    lam, phi0 = csff.contour_bound_state(c["v1"], c["h"], g, -1.0)
    kn = math.sqrt(2.0 * (E - lam.real))
    X = [csff.contour_regular_solution(c["v1"], c["h"], g, kn)]
    Y = [phi0]
    al = PW.alpha_midpoints(16)
    k = math.sqrt(2.0 * E)
    for a in al:
        X.append(csff.contour_regular_solution(c["v1"], c["h"], g, k * math.sin(a)))
        Y.append(csff.contour_regular_solution(c["v1"], c["h"], g, k * math.cos(a)))
    m = n - 2
    amp = plan.separable_sum(dev(np.stack(X)).reshape(-1, m), dev(np.stack(Y)).reshape(-1, m), dev(c["f"]),
                             dev(c["w"]), u).cpu().numpy()
    uo = PW.solve(E, n)
    so, _ = PW.single_amplitude(E, uo, n)
    fo = PW.double_amplitudes(E, uo, al, n)
    assert abs(amp[0] - so) <= 1e-8 * abs(so)
    assert np.abs(amp[1:] - fo).max() <= 1e-8 * np.abs(fo).max()
    plan.close()
