"""3D path (7-point stencil, trilinear transfers, sum-factorised far field)
against the oracle on a small grid, and the full 257^3 sixteen-direction case
through properties that hold at any size."""
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


def test_3d_mixed_far_field_on_the_full_angle_grid(csff):
    c = W.big_3d(n=33, n_rhs=2)
    c["opts"]["precision"] = "mixed"
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    eta = c["eta"]
    u = torch.zeros(2 * plan.N, dtype=torch.complex128, device="cuda")
    st, infos = plan.solve(eta, u)
    assert st == csff.OK and all(i["rel_res"] <= 1e-8 for i in infos)
    al = c["alphas"]
    F = torch.zeros(2 * len(al), dtype=torch.complex128, device="cuda")
    plan.far_field(eta, u, al, F)
    Fg = F.cpu().numpy().reshape(2, -1)
    for r in range(2):
        ug = u[r * plan.N:(r + 1) * plan.N].cpu().numpy().reshape((p.m,) * 3)
        # same solution: rounding-level agreement of the contraction
        m, e2, tn = O.far_field(p, ug, eta[r], al, return_terms_norm=True)
        Fo = O.far_field_value(m, e2)
        assert np.abs(Fg[r] - Fo).max() <= 1e-12 * (tn * 2.0 ** e2).max()
        # against the oracle's own solve, over the well-conditioned directions
        res = O.mg_solve(p, O.rhs(p, eta[r]), O.opts_from_dict(c["opts"]))
        m2, e22, tn2 = O.far_field(p, res.u, eta[r], al, return_terms_norm=True)
        F2 = O.far_field_value(m2, e22)
        kappa = tn2 / np.maximum(np.abs(m2), 1e-300)
        cone = kappa * 1e-8 <= 1e-6
        assert cone.sum() >= 50
        assert np.linalg.norm(Fg[r][cone] - F2[cone]) <= 1e-5 * np.linalg.norm(F2[cone])


def test_3d_full_size_sixteen_directions(csff):
    """257^3 on [-15,15]^3, k = 4, 16 incident directions, mixed precision:
    every solve meets 1e-8 (re-checked with the oracle's operator on one
    direction) and the maps obey reciprocity F(-eta_j; eta_i) = F(-eta_i; eta_j)
    over the directions where the sum is well conditioned."""
    c = W.big_3d(n=257, n_rhs=16)
    c["opts"]["precision"] = "mixed"
    plan = csff.Plan(c["problem"], c["opts"])
    eta = c["eta"]
    u = torch.zeros(16 * plan.N, dtype=torch.complex128, device="cuda")
    st, infos = plan.solve(eta, u)
    assert st == csff.OK and all(i["rel_res"] <= 1e-8 for i in infos)
    p = O.problem_from_dict(c["problem"])
    u0 = u[:plan.N].cpu().numpy().reshape((p.m,) * 3)
    b0 = O.rhs(p, eta[0])
    lv = O.make_level(p, p.n)
    assert O.norm2(O.residual(lv, u0, b0)) <= 1.01e-8 * O.norm2(b0)
    del u0, b0, lv
    # reciprocity on the 16 x 16 map of outgoing -eta_j for incident eta_i
    F = torch.zeros(16 * 16, dtype=torch.complex128, device="cuda")
    Fe = torch.zeros(16 * 16, dtype=torch.int32, device="cuda")
    plan.far_field(eta, u, -eta, F, Fe)
    M = (F.cpu().numpy() * 2.0 ** Fe.cpu().numpy().astype(np.float64)).reshape(16, 16)
    scale = np.abs(np.diag(M)).max()   # forward scattering amplitudes set the scale
    ok = 0
    for i in range(16):
        for j in range(16):
            if abs(M[i, j]) > 1e-3 * scale:
                ok += 1
                assert abs(M[i, j] - M[j, i]) <= 1e-5 * abs(M[i, j])
    assert ok >= 16
    plan.close()


def _maps(csff, plan, c, u, mode):
    plan.set_far_field_mode(mode)
    al = c["alphas"]
    nr = len(c["eta"])
    F = torch.zeros(nr * len(al), dtype=torch.complex128, device="cuda")
    E = torch.zeros(nr * len(al), dtype=torch.int32, device="cuda")
    plan.far_field(c["eta"], u, al, F, E)
    return (F.cpu().numpy() * 2.0 ** E.cpu().numpy().astype(np.float64)).reshape(nr, len(al))


def test_3d_tensor_core_far_field_against_oracle(csff):
    """Tensor-core z-contraction (four-way BF16 split of each operand, ten
    products, FP32 accumulation over 32 z-nodes, double-float sums across
    them): per angle within 2^-24 sum|terms| of the oracle on the same
    solution (2^-25.5 measured), and within the 1e-5 relative L2 target over
    the 64 x 32 map."""
    c = W.big_3d(n=65, n_rhs=2)
    c["opts"]["precision"] = "mixed"
    plan = csff.Plan(c["problem"], c["opts"])
    p = O.problem_from_dict(c["problem"])
    u = torch.zeros(2 * plan.N, dtype=torch.complex128, device="cuda")
    plan.solve(c["eta"], u)
    Ft = _maps(csff, plan, c, u, csff.FF_TC_BF16X4)
    for r in range(2):
        ug = u[r * plan.N:(r + 1) * plan.N].cpu().numpy().reshape((p.m,) * 3)
        m, e2, tn = O.far_field(p, ug, c["eta"][r], c["alphas"], return_terms_norm=True)
        Fo = O.far_field_value(m, e2)
        assert np.all(np.abs(Ft[r] - Fo) <= 2.0 ** -24 * tn * 2.0 ** e2)
        assert np.linalg.norm(Ft[r] - Fo) <= 1e-5 * np.linalg.norm(Fo)
    plan.close()


def test_3d_tensor_core_falls_back_when_the_range_is_too_wide(csff):
    """k = 8 on [-15,15]^3 with u = 0: the phase rows span e^{+-60} and the
    columns of g = chi u_in as much, so the device-side range check keeps the
    FP64 kernel; the maps are then identical bit for bit."""
    c = W.big_3d(n=33, n_rhs=1)
    c["problem"]["k"] = 8.0
    c["opts"]["precision"] = "mixed"
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")      # g = chi u_in
    F64 = _maps(csff, plan, c, u, csff.FF_FP64)
    Ft = _maps(csff, plan, c, u, csff.FF_TC_BF16X4)
    assert np.array_equal(F64, Ft)
    plan.close()


def test_3d_full_size_tensor_core_maps(csff):
    """257^3, 16 directions: the tensor-core maps against the FP64 maps of the
    same solutions.  Relative L2 per map is about 2^-26 times the map's
    condition number (four-term splits, FP32 accumulation over 32 z-nodes,
    double-float across chunks): 1.1e-6 to 5.7e-6 measured; every map within
    the 1e-5 target."""
    c = W.big_3d(n=257, n_rhs=16)
    c["opts"]["precision"] = "mixed"
    plan = csff.Plan(c["problem"], c["opts"])
    u = torch.zeros(16 * plan.N, dtype=torch.complex128, device="cuda")
    plan.solve(c["eta"], u)
    F64 = _maps(csff, plan, c, u, csff.FF_FP64)
    Ft = _maps(csff, plan, c, u, csff.FF_TC_BF16X4)
    rel = np.linalg.norm(Ft - F64, axis=1) / np.linalg.norm(F64, axis=1)
    assert rel.max() <= 1e-5
    plan.close()
