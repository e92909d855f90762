"""Pins of the CPU oracle against facts fixed by the paper and by mathematics
(not by re-typing the oracle's own formulas).  CPU only."""
import math
import os

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.sparse.linalg as spla

import oracle.csff_oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _prob(dim=2, n=17, R=5.0, gamma=math.pi / 6, k=2.0, gs=None):
    gs = [O.Gaussian(-0.5, 2.0)] if gs is None else gs
    return O.Problem(dim, n, -R, R, gamma, k, gs)


# ---------------------------------------------------------------------------
# Table 1 and eq. (mingammajac): printed values
# ---------------------------------------------------------------------------
def test_table1_gamma_from_ecs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_gamma_from_ecs.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 6
    for den, gdeg in rows:
        g = math.degrees(O.gamma_from_ecs(math.pi / int(den)))
        assert abs(g - float(gdeg)) <= 0.05 + 1e-9, (den, g, gdeg)


def test_min_gamma_is_13_degrees():
    # Sec. 3.3: beta_min = 0.5 gives gamma >= 0.23 rad, about 13 degrees.
    g = O.min_gamma(0.5)
    assert abs(g - 0.23) < 0.005 and round(math.degrees(g)) == 13


def test_csl_shift_of_30_degrees():
    # eq. (csl): e^{i 2 gamma} = alpha + i beta; at gamma = 30 deg beta = sin 60 deg.
    s = O.csl_shift(math.pi / 6)
    assert abs(s.real - 0.5) < 1e-15 and abs(s.imag - math.sqrt(3) / 2) < 1e-15


# ---------------------------------------------------------------------------
# The stencil: exact eigenpairs of the Dirichlet Laplacian
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 9), (2, 17), (3, 9)])
def test_operator_on_sine_eigenvectors(dim, n):
    """With constant chi = chi0 the discrete sine modes are eigenvectors:
    A v = (e^{-2i gamma}/h^2 * sum_c 4 sin^2(pi a_c / (2(n-1))) - k^2 (1 + chi0)) v."""
    chi0 = 0.3 - 0.2j
    p = _prob(dim, n, gs=[O.Gaussian(chi0, 1e300)])   # width -> infinity: chi == chi0
    lv = O.make_level(p, n)
    m = n - 2
    rng = np.random.default_rng(1)
    A_sp = O.assemble_matrix(lv)
    for _ in range(4):
        a = rng.integers(1, n - 1, size=dim)
        v = np.ones((m,) * dim)
        lam = 0.0
        for c in range(dim):
            i = np.arange(1, n - 1)
            shape = [1] * dim
            shape[dim - 1 - c] = m
            v = v * np.sin(math.pi * a[c] * i / (n - 1)).reshape(shape)
            lam += 4 * math.sin(math.pi * a[c] / (2 * (n - 1))) ** 2
        mu = np.exp(-2j * p.gamma) / p.h ** 2 * lam - p.k ** 2 * (1 + chi0)
        Av = O.apply_A(lv, v)
        assert np.abs(Av - mu * v).max() <= 1e-12 * np.abs(mu)
        Av2 = (A_sp @ v.ravel()).reshape(v.shape)
        assert np.abs(Av2 - mu * v).max() <= 1e-12 * np.abs(mu)


def test_operator_is_complex_symmetric():
    """A^T = A (not Hermitian): the property behind far-field reciprocity."""
    p = _prob(2, 9, gs=[O.Gaussian(-0.5, 2.0, (0.7, -0.3, 0.0))])
    A = O.assemble_matrix(O.make_level(p, 9)).toarray()
    assert np.abs(A - A.T).max() == 0.0
    assert np.abs(A - A.conj().T).max() > 1e-3


def test_chi_radial_closed_form():
    """For a centred Gaussian chi(x e^{i g}) = A exp(-|x|^2 e^{2 i g} / w)."""
    p = _prob(3, 9, R=4.0, gs=[O.Gaussian(-1.5 + 0.5j, 3.0)])
    chi = O.chi_at_nodes(p)
    x = O.interior_coords(9, -4.0, 4.0)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ref = (-1.5 + 0.5j) * np.exp(-(X ** 2 + Y ** 2 + Z ** 2) * np.exp(2j * p.gamma) / 3.0)
    assert np.abs(chi - ref).max() <= 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# Constant coefficients: exact solution by the discrete sine transform
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, 33), (3, 17)])
def test_direct_and_vcycle_match_sine_transform_solution(dim, n):
    chi0 = -0.4 + 0.1j
    p = _prob(dim, n, R=6.0, k=1.5, gs=[O.Gaussian(chi0, 1e300)])
    b = W.rand_complex((n - 2,) * dim, seed=7)
    m = n - 2
    lam = 4 * np.sin(math.pi * np.arange(1, m + 1) / (2 * (n - 1))) ** 2
    L = sum(np.meshgrid(*([lam] * dim), indexing="ij"))
    mu = np.exp(-2j * p.gamma) / p.h ** 2 * L - p.k ** 2 * (1 + chi0)
    u_exact = sfft.idstn(sfft.dstn(b, type=1) / mu, type=1)
    u_dir = O.direct_solve(p, b)
    assert np.linalg.norm(u_dir - u_exact) <= 1e-12 * np.linalg.norm(u_exact)
    opts = O.MGOptions(smoother="jacobi", nu1=2, nu2=2, coarsest_n=5, rel_tol=1e-12)
    res = O.mg_solve(p, b, opts)
    assert res.converged
    assert np.linalg.norm(res.u - u_exact) <= 1e-9 * np.linalg.norm(u_exact)


# ---------------------------------------------------------------------------
# Smoothers: brute-force pure-Python loops on tiny grids
# ---------------------------------------------------------------------------
def _py_point_residual(lv, u, b, idx):
    d = lv.dim
    s = 0.0
    for ax in range(d):
        for sgn in (-1, 1):
            j = list(idx)
            j[ax] += sgn
            if 0 <= j[ax] < lv.m:
                s += u[tuple(j)]
    au = lv.c * (2 * d * u[idx] - s) - lv.q[idx] * u[idx]
    return b[idx] - au


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 5)])
def test_rbgs_matches_sequential_loop(dim, n):
    p = _prob(dim, n, gs=[O.Gaussian(-0.5, 2.0, (0.3, 0.0, -0.2))])
    lv = O.make_level(p, n)
    u0 = W.rand_complex((n - 2,) * dim, seed=3)
    b = W.rand_complex((n - 2,) * dim, seed=4)
    u = u0.copy()
    for colour in (0, 1):             # red (even node-index sum) first, in place
        for idx in np.ndindex(*u.shape):
            if (sum(idx) + dim) % 2 == colour:
                u[idx] = u[idx] + _py_point_residual(lv, u, b, idx) / lv.diag[idx]
    assert np.abs(O.rbgs(lv, u0, b) - u).max() <= 1e-13 * np.abs(u).max()


def test_jacobi_matches_loop():
    n, dim = 9, 2
    p = _prob(dim, n)
    lv = O.make_level(p, n)
    u0 = W.rand_complex((n - 2,) * dim, seed=5)
    b = W.rand_complex((n - 2,) * dim, seed=6)
    ref = np.empty_like(u0)
    for idx in np.ndindex(*u0.shape):
        ref[idx] = u0[idx] + 0.6 * _py_point_residual(lv, u0, b, idx) / lv.diag[idx]
    assert np.abs(O.jacobi(lv, u0, b, 0.6) - ref).max() <= 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# Grid transfers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_is_2d_times_fw_transpose(dim):
    mc = 3 if dim == 3 else 7
    mf = 2 * mc + 1
    r = W.rand_complex((mf,) * dim, seed=11)
    e = W.rand_complex((mc,) * dim, seed=12)
    lhs = np.vdot(e, O.restrict_fw(r)) * 2 ** dim
    rhs = np.vdot(O.prolong(e), r)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def _parabola(n):
    """f(i) = i (n-1-i): zero on both boundary nodes, second difference -2."""
    i = np.arange(n, dtype=float)
    return i * (n - 1 - i)


@pytest.mark.parametrize("dim", [2, 3])
def test_transfers_on_separable_parabola(dim):
    """1D facts for f(i) = i(N-i) in units of the fine spacing: full weighting
    gives f - 1/2 (times 1/4 of the second difference, -2 per fine step);
    linear interpolation misses the coarse parabola by exactly 1 at midpoints
    (H^2/4 in units where H = 2).  Tensor products give the d-dimensional
    values."""
    nc = 9
    nf = 2 * nc - 1
    ff = _parabola(nf)                     # fine-grid values of f
    fw1 = ff[2:-2:2] - 0.5                 # FW at the coarse interior nodes
    pr1 = ff.copy()
    pr1[1::2] -= 1.0                       # interpolated coarse samples
    def outer(vs):
        out = vs[0]
        for v in vs[1:]:
            out = np.multiply.outer(v, out)
        return out
    r = outer([ff[1:-1]] * dim)
    assert np.abs(O.restrict_fw(r) - outer([fw1] * dim)).max() < 1e-10
    e = outer([ff[2:-2:2]] * dim)          # coarse interior samples of f
    assert np.abs(O.prolong(e) - outer([pr1[1:-1]] * dim)).max() < 1e-10


# ---------------------------------------------------------------------------
# Solver: V-cycle reaches the sparse direct solution on variable chi
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n,smoother", [(2, 17, "jacobi"), (2, 33, "rbgs"), (3, 9, "rbgs"),
                                            (3, 17, "jacobi")])
def test_vcycle_converges_to_direct_solve(dim, n, smoother):
    p = _prob(dim, n, R=6.0, k=1.5, gs=[O.Gaussian(-0.5, 2.0)])
    b = O.rhs(p, [1.0, 0.0, 0.0][:dim])
    opts = O.MGOptions(smoother=smoother, omega=2 / 3 if smoother == "jacobi" else 1.0,
                       nu1=1, nu2=1, coarsest_n=5, rel_tol=1e-11)
    res = O.mg_solve(p, b, opts)
    # omega = 2/3 Jacobi is a weaker smoother in 3D (its optimum there is 6/7)
    assert res.converged and res.conv_factor < (0.7 if (dim, smoother) == (3, "jacobi") else 0.5)
    ud = O.direct_solve(p, b)
    assert np.linalg.norm(res.u - ud) <= 1e-8 * np.linalg.norm(ud)


def test_small_2d_case_converges():
    c = W.small_2d()
    p = O.problem_from_dict(c["problem"])
    res = O.mg_solve(p, O.rhs(p, c["eta"][0]), O.opts_from_dict(c["opts"]))
    assert res.converged and res.history[-1] <= 1e-10
    assert all(h1 < h0 for h0, h1 in zip(res.history, res.history[1:]))


# ---------------------------------------------------------------------------
# Far field
# ---------------------------------------------------------------------------
def test_chi_zero_gives_zero():
    p = _prob(2, 17, gs=[O.Gaussian(0.0, 2.0)])
    b = O.rhs(p, [1.0, 0.0])
    assert np.all(b == 0)
    res = O.mg_solve(p, b, O.MGOptions())
    assert np.all(res.u == 0)
    m, e = O.far_field(p, res.u, [1.0, 0.0], W.angle_set_2d(8))
    assert np.all(m == 0)


@pytest.mark.parametrize("dim,n,R,k", [(2, 129, 20.0, 2.0), (3, 65, 12.0, 1.0)])
def test_born_closed_form(dim, n, R, k):
    """Weak potential: (F(A) - F(-A))/2 is the first Born term up to O(A^3),
    which for chi = A exp(-|x|^2/w) is k^2 A (pi w)^{d/2} exp(-w k^2 |eta-alpha|^2 / 4).
    The contour sum of the analytic integrand equals the real-axis integral
    once the box truncation (e^{-R^2 cos 2g / w + k sin g |eta-alpha| R}) and
    the aliasing of the rotated Gaussian (spacing h) are below 1e-9."""
    w, A = 2.0, 1e-4
    eta = [1.0, 0.0, 0.0][:dim]
    al = W.angle_set_2d(16) if dim == 2 else W.angle_set_3d(6, 4)
    Fs = []
    for a in (A, -A):
        p = O.Problem(dim, n, -R, R, math.pi / 6, k, [O.Gaussian(a, w)])
        b = O.rhs(p, eta)
        if dim == 2:
            u = O.direct_solve(p, b)
        else:
            u = O.mg_solve(p, b, O.MGOptions(smoother="rbgs", rel_tol=1e-10)).u
        Fs.append(O.far_field_value(*O.far_field(p, u, eta, al)))
    Fsym = (Fs[0] - Fs[1]) / 2
    Fb = np.array([O.born_far_field(k, A, w, dim, eta, a) for a in al])
    assert np.abs(Fsym - Fb).max() <= 5e-8 * np.abs(Fb).max()


def test_far_field_of_incident_part_against_high_precision_sum():
    """u := 0 leaves the separable sum k^2 A e^{i d g} h^d prod_c S_c(alpha),
    S_c = sum_i exp(-z_i^2/w + i k (eta_c - alpha_c) z_i), z_i = x_i e^{i g};
    evaluated here independently in 40-digit arithmetic.  Pins the phase sign,
    Jacobian and weights also where the sum is badly conditioned (30 degrees,
    k = 2 on [-10, 10]^2)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    c = W.small_2d(n=33)
    p = O.problem_from_dict(c["problem"])
    eta = c["eta"][0]
    al = W.angle_set_2d(12)
    m, e, tn = O.far_field(p, np.zeros((31, 31), complex), eta, al, return_terms_norm=True)
    F = O.far_field_value(m, e)
    g = mp.mpf(p.gamma)
    rot = mp.expj(g)
    xs = [mp.mpf(p.lo) + i * mp.mpf(p.h) for i in range(1, p.n - 1)]
    A, w = p.gaussians[0].amp, p.gaussians[0].width
    for a, alpha in enumerate(al):
        S = []
        for cc in range(2):
            q = mp.mpf(p.k) * (mp.mpf(eta[cc]) - mp.mpf(alpha[cc]))
            S.append(mp.fsum(mp.exp(-(x * rot) ** 2 / w + 1j * q * x * rot) for x in xs))
        ref = mp.mpf(p.k) ** 2 * mp.mpc(A) * mp.expj(2 * g) * mp.mpf(p.h) ** 2 * S[0] * S[1]
        ref = complex(ref)
        assert abs(F[a] - ref) <= 1e-14 * tn[a] * 2.0 ** e[a] + 1e-300


def test_mirror_symmetry():
    """eta = +x and chi even in y: F(a_x, a_y) = F(a_x, -a_y)."""
    p = _prob(2, 33, R=8.0, k=1.5, gs=[O.Gaussian(-0.5, 2.0, (0.8, 0.0, 0.0))])
    u = O.direct_solve(p, O.rhs(p, [1.0, 0.0]))
    al = W.angle_set_2d(24)
    F = O.far_field_value(*O.far_field(p, u, [1.0, 0.0], al))
    Fm = O.far_field_value(*O.far_field(p, u, [1.0, 0.0], al * np.array([1.0, -1.0])))
    assert np.abs(F - Fm).max() <= 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("dim,n", [(2, 33), (3, 9)])
def test_reciprocity(dim, n):
    """A is complex symmetric and the weights are uniform, so the discrete map
    satisfies F(alpha; eta) = F(-eta; -alpha) exactly."""
    p = _prob(dim, n, R=6.0, k=1.5, gs=[O.Gaussian(-0.7, 2.0, (0.5, -0.4, 0.3))])
    dirs = W.angle_set_2d(6) if dim == 2 else W.angle_set_3d(4, 2)
    F = {}
    for i, eta in enumerate(dirs):
        u = O.direct_solve(p, O.rhs(p, eta))
        F[i] = O.far_field_value(*O.far_field(p, u, eta, -dirs))
    # F(alpha_j; eta_i) with alpha_j = -dirs[j]; reciprocity: F(-d_j; d_i) = F(-d_i; d_j)
    for i in range(len(dirs)):
        for j in range(len(dirs)):
            assert abs(F[i][j] - F[j][i]) <= 1e-11 * max(abs(F[i][j]), 1e-30)


def test_contour_independence_second_order():
    """eq. (I2complex) holds for any rotation: maps at 20 and 30 degrees differ
    only by the O(h^2) discretisation error (ratio about 4 per grid halving)."""
    al = W.angle_set_2d(32)
    diffs = []
    for n in (65, 129):
        F = {}
        for gd in (20, 30):
            p = O.Problem(2, n, -20, 20, gd * math.pi / 180, 1.0, [O.Gaussian(-0.5, 2.0)])
            u = O.direct_solve(p, O.rhs(p, [1.0, 0.0]))
            F[gd] = O.far_field_value(*O.far_field(p, u, [1.0, 0.0], al))
        diffs.append(np.linalg.norm(F[20] - F[30]) / np.linalg.norm(F[30]))
    assert diffs[1] < 2e-3
    assert 3.0 < diffs[0] / diffs[1] < 5.0


def test_far_field_extended_range():
    """Terms beyond the FP64 range (k = 40 on [-20,20]^2 at 30 degrees) come
    back as finite mantissa/exponent pairs; where the plain sum is representable
    the two agree."""
    c = W.mixed_2d(40.0, n=129)
    p = O.problem_from_dict(c["problem"])
    al = W.angle_set_2d(8)
    m, e = O.far_field(p, np.zeros((127, 127), complex), c["eta"][0], al)
    assert np.all(np.isfinite(m)) and e.max() > 1024
    c = W.mixed_2d(5.0, n=129)
    p = O.problem_from_dict(c["problem"])
    m, e = O.far_field(p, np.zeros((127, 127), complex), c["eta"][0], al)
    F = O.far_field_value(m, e)
    g = O.chi_at_nodes(p) * O.u_incident(p, c["eta"][0])
    X = O._axis_coords(2, p.n, p.lo, p.hi)
    for a, alpha in enumerate(al):
        P = np.exp(-1j * p.k * np.exp(1j * p.gamma) * (alpha[0] * X[0] + alpha[1] * X[1]))
        ref = p.k ** 2 * np.exp(2j * p.gamma) * p.h ** 2 * np.sum(P * g)
        assert abs(F[a] - ref) <= 1e-12 * np.sum(np.abs(P * g)) * p.k ** 2 * p.h ** 2


def test_rhs_stays_finite_for_oblique_incidence_at_large_k():
    """k = 52, w = 1 on [-20,20]^2 with eta at 45 degrees: |u_in| alone reaches
    e^{k sin(g) R sqrt 2} = e^{735} (beyond FP64) at the upstream corner, while
    chi u_in peaks at e^{338} (t* = k sin(g) w / (2 cos 2g) = 26 along -eta);
    the source is evaluated without overflow and equals the product of the two
    factors wherever those fit."""
    p = O.Problem(2, 65, -20.0, 20.0, math.pi / 6, 52.0, [O.Gaussian(-1.0, 1.0)])
    eta = [math.sqrt(0.5), math.sqrt(0.5)]
    b = O.rhs(p, eta)
    assert np.all(np.isfinite(b))
    assert np.log(np.abs(b).max() / p.k ** 2) <= 338.5
    with np.errstate(over="ignore", invalid="ignore"):
        prod = p.k ** 2 * O.chi_at_nodes(p) * O.u_incident(p, eta)
    fin = np.isfinite(prod)
    assert fin.sum() > 0.5 * fin.size and not fin.all()
    # exponents up to ~340 and phases up to ~1500 rad: both evaluations round
    # them at ~1e-16 relative, i.e. ~1e-13 relative in the values
    assert np.all(np.abs(b[fin] - prod[fin]) <= 1e-10 * np.abs(prod[fin]) + 1e-14 * np.abs(b).max())


# ---------------------------------------------------------------------------
# GMRES(m) smoothing step (Sec. 3.3, Tables 2-3): pinned by what GMRES is --
# the minimiser of the residual over the shifted Krylov space -- computed here
# by brute force, by the full-space case and by the m = 1 closed form
# ---------------------------------------------------------------------------
def _gmres_level(n=17, dim=2):
    c = W.paper_gmres(dim=dim, k=1.0, n=n)
    p = O.problem_from_dict(c["problem"])
    return O.make_hierarchy(p, 5)[0]


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_gmres_step_is_the_krylov_least_squares_minimiser(m):
    lv = _gmres_level(17)
    shp = (lv.m,) * 2
    u = W.rand_complex(shp, 41)
    b = W.rand_complex(shp, 42)
    r0 = O.residual(lv, u, b)
    # Krylov basis r0, A r0, ..., A^{m-1} r0 (unorthogonalised) and the dense
    # least-squares problem min_c || r0 - A K c ||
    K = [r0]
    for _ in range(m - 1):
        K.append(O.apply_A(lv, K[-1]))
    AK = np.stack([O.apply_A(lv, v).ravel() for v in K], axis=1)
    cvec = np.linalg.lstsq(AK, r0.ravel(), rcond=None)[0]
    x_bf = u + sum(ci * v for ci, v in zip(cvec, K))
    x = O.gmres_smooth(lv, u, b, m)
    assert np.abs(x - x_bf).max() <= 1e-9 * np.abs(x_bf - u).max()
    # and its residual is no larger than that of any other point of the space
    rng = np.random.default_rng(7)
    rx = O.norm2(O.residual(lv, x, b))
    for _ in range(5):
        pert = cvec + 1e-3 * (rng.standard_normal(m) + 1j * rng.standard_normal(m)) * np.abs(cvec).max()
        xp = u + sum(ci * v for ci, v in zip(pert, K))
        assert rx <= O.norm2(O.residual(lv, xp, b)) * (1 + 1e-12)


def test_gmres_over_the_whole_space_is_the_direct_solve():
    # 9 unknowns: GMRES(9) spans the whole space, so one step solves exactly
    c = W.paper_gmres(dim=2, k=1.0, n=5)
    p = O.problem_from_dict(c["problem"])
    lv = O.make_hierarchy(p, 5)[0]
    b = W.rand_complex((3, 3), 43)
    u0 = W.rand_complex((3, 3), 44)
    A = O.assemble_matrix(lv).toarray()
    x_ref = np.linalg.solve(A, b.ravel()).reshape(3, 3)
    x = O.gmres_smooth(lv, u0, b, 9)
    assert np.abs(x - x_ref).max() <= 1e-10 * np.abs(x_ref).max()


def test_gmres1_is_the_minimal_residual_step():
    # m = 1: u + a r with a = (A r, r) / (A r, A r), the one-dimensional minimiser
    lv = _gmres_level(17)
    shp = (lv.m,) * 2
    u = W.rand_complex(shp, 45)
    b = W.rand_complex(shp, 46)
    r = O.residual(lv, u, b)
    Ar = O.apply_A(lv, r)
    a = np.vdot(Ar, r) / np.vdot(Ar, Ar)
    x = O.gmres_smooth(lv, u, b, 1)
    assert np.abs(x - (u + a * r)).max() <= 1e-12 * np.abs(a * r).max()


def test_gmres_leaves_an_exact_solution_alone():
    lv = _gmres_level(9)
    x = W.rand_complex((lv.m, lv.m), 47)
    b = O.apply_A(lv, x)
    out = O.gmres_smooth(lv, x, b, 3)
    assert np.abs(out - x).max() <= 1e-12 * np.abs(x).max()


def test_gmres_vcycle_stable_where_gauss_seidel_is_not():
    # Sec. 3.3: with omega-Jacobi / Gauss-Seidel smoothing the rotation must be
    # at least about 13 degrees; with GMRES(m) about 10 degrees suffices.  On
    # eq. (chi2D) at 9.9 degrees the red-black V(1,1) cycle diverges and the
    # GMRES(3) V(1,1) cycle converges with factors in the range the paper
    # reports for its V(1,1)/GMRES(3) runs (Table 2: 0.01-0.33).
    c = W.paper_gmres(dim=2, k=1.0, n=65)
    p = O.problem_from_dict(c["problem"])
    b = O.rhs(p, c["eta"][0])
    og = O.opts_from_dict(c["opts"])
    rg = O.mg_solve(p, b, og)
    assert rg.converged and rg.cycles <= 15 and rg.conv_factor <= 0.35
    orb = O.opts_from_dict(dict(c["opts"], smoother="rbgs", max_cycles=12))
    rr = O.mg_solve(p, b, orb)
    assert not rr.converged and rr.history[-1] > 1.0


def _table2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table2_vcycle_gmres3.txt"))
            if l.strip() and not l.startswith("#")]
    return [(float(k), int(n), int(c), float(f)) for k, n, c, f in rows]


@pytest.mark.parametrize("pts", [16, 32])
def test_gmres_vcycle_reproduces_table2(pts):
    # Table 2's V(1,1)/GMRES(3) cycle counts and factors on the 16^3 and 32^3
    # grids (eq. chi3D, 9.9 degrees, 1e-6): the oracle's cycle counts agree to
    # within two cycles and its factors to within 0.07 for every k0
    rows = [r for r in _table2() if r[1] == pts]
    assert len(rows) == 5
    for k, n, cyc, fac in rows:
        c = W.paper_gmres(dim=3, k=k, n=n + 1)
        p = O.problem_from_dict(c["problem"])
        b = O.rhs(p, c["eta"][0])
        r = O.mg_solve(p, b, O.opts_from_dict(c["opts"]))
        assert r.converged
        assert abs(r.cycles - cyc) <= 2, (k, n, r.cycles, cyc)
        assert abs(r.conv_factor - fac) <= 0.07, (k, n, r.conv_factor, fac)


# ---------------------------------------------------------------------------
# Full multigrid (Sec. 4, FMG paragraph; Table 3)
# ---------------------------------------------------------------------------
def _fmg_case(dim, n, k=2.0):
    if dim == 2:
        c = W.small_2d(n=n)
        c["problem"]["k"] = k
        c["opts"].update(smoother="rbgs", nu1=1, nu2=1, coarsest_n=5, rel_tol=1e-9, max_cycles=60)
    else:
        c = W.paper_gmres(dim=3, k=1.0, n=n)
        c["opts"].update(rel_tol=1e-8, max_cycles=60)
    p = O.problem_from_dict(c["problem"])
    return p, O.opts_from_dict(c["opts"]), O.rhs(p, c["eta"][0])


@pytest.mark.parametrize("dim,n", [(2, 33), (2, 65), (3, 17)])
def test_fmg_reaches_the_direct_solution(dim, n):
    """Every level meets the tolerance and the finest iterate agrees with a
    sparse direct solve to within the tolerance's error bound."""
    p, o, b = _fmg_case(dim, n)
    res = O.fmg_solve(p, b, o)
    assert res.converged and len(res.level_cycles) == len(O.make_hierarchy(p, o.coarsest_n)) - 1
    assert all(h[-1] <= o.rel_tol for h in res.level_history)
    ud = O.direct_solve(p, b)
    A = O.assemble_matrix(O.make_level(p, p.n))
    # ||u - u*|| <= ||A^-1|| ||r||: bound ||A^-1|| by a few inverse-power steps
    x = W.rand_complex(A.shape[0], 5)
    lu = spla.splu(A.tocsc())
    for _ in range(30):
        x = lu.solve(x)
        nrm = np.linalg.norm(x)
        x /= nrm
    err = np.linalg.norm(res.u - ud) / np.linalg.norm(ud)
    assert err <= 2.0 * nrm * o.rel_tol * np.linalg.norm(b) / np.linalg.norm(ud)


def test_fmg_without_cycles_is_the_interpolated_coarse_solution():
    """With no V-cycles the two-level FMG returns P A_c^{-1} FW(b): the coarse
    problem solved by an independent sparse direct solve, then interpolated."""
    p, o, b = _fmg_case(2, 9)
    o.max_cycles = 0
    res = O.fmg_solve(p, b, o)
    pc = O.Problem(2, 5, p.lo, p.hi, p.gamma, p.k, p.gaussians)
    uc = spla.spsolve(O.assemble_matrix(O.make_level(pc, 5)).tocsc(), O.restrict_fw(b).ravel()).reshape(3, 3)
    ref = O.prolong(uc)
    assert res.level_cycles == [0]
    assert np.abs(res.u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fmg_on_a_single_level_is_the_direct_solve():
    p, o, b = _fmg_case(2, 5)
    res = O.fmg_solve(p, b, o)
    assert res.level_cycles == []
    ref = spla.spsolve(O.assemble_matrix(O.make_level(p, 5)).tocsc(), b.ravel()).reshape(b.shape)
    assert np.abs(res.u - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("pts", [16, 32])
def test_fmg_finest_level_needs_no_more_cycles_than_vcycles_from_zero(pts):
    """Table 3's setting (eq. chi3D, 9.9 degrees, V(1,1)/GMRES(3), 1e-6): the
    nested iteration's finest level needs at most the V-cycles the iteration
    from zero needs (Table 2's setting).  Table 3 prints 2-4 fewer finest-level
    cycles than Table 2 on these grids; this reading of the FMG saves at most
    one (the paper does not give its coarse right-hand sides or the reference
    of its per-level tolerance), so the printed counts are context, not a pin."""
    for k in (0.25, 0.5, 1.0, 2.0, 4.0):
        c = W.paper_gmres(dim=3, k=k, n=pts + 1)
        p = O.problem_from_dict(c["problem"])
        o = O.opts_from_dict(c["opts"])
        b = O.rhs(p, c["eta"][0])
        f = O.fmg_solve(p, b, o)
        v = O.mg_solve(p, b, o)
        assert f.converged and v.converged
        assert f.cycles <= v.cycles, (k, f.level_cycles, v.cycles)
