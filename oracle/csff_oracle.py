"""Plain, slow, FP64 CPU oracle for the complex-contour multigrid far-field method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

Method (Cools, Reps & Vanroose, "An efficient multigrid calculation of the Far
Field map for Helmholtz and Schroedinger equations"):

* Sec. 2.1, eq. (helmholtz_in): scattered wave u solves
  (-Delta - k^2(1+chi)) u = k^2 chi u_in, with u_in = exp(i k eta.x).
* Sec. 3.1, eq. (I2complex): the far-field integral is taken over the rotated
  contour z = x e^{i gamma}; the integrand picks up the Jacobian e^{i d gamma}
  in d dimensions and chi, u_in, u are evaluated at complex z.
* Sec. 3.2, eq. (csg) and the 1D stencil of Sec. 5.2: finite differences with
  the complex spacing h e^{i gamma} give the operator
  A u = e^{-2i gamma} (2d u - sum_nbr u) / h^2 - k^2 (1 + chi(z)) u.
* Sec. 4: V(nu1, nu2) cycles with omega-Jacobi (or Gauss-Seidel) smoothing,
  full-weighting restriction and bi/trilinear interpolation, iterated to a
  residual-reduction tolerance; Sec. 3.3 and Tables 2-3: GMRES(m) cycles as
  the smoother at rotation angles near 10 degrees.
* eq. (FFmap) with (I2complex): F(alpha) = int e^{-i k z.alpha}
  k^2 chi(z) (u_in(z) + u(z)) dz, evaluated with uniform weights h^d over the
  interior nodes (the paper allows any quadrature, Sec. 4).

Readings taken where the paper is silent or garbled (each repeated in the
design notes):
* the rotation angle is called gamma (the paper's theta is the ECS angle);
* eq. (csg) is read with the sign of the Sec. 5.2 stencil: A = e^{-2i gamma} L/h^2 - k^2(1+chi);
* homogeneous Dirichlet values on the boundary ring of the rotated box;
* the d-dimensional Jacobian is e^{i d gamma};
* chi(z) = A exp(-sum_c (z_c - center_c)^2 / w), the analytic continuation of
  the real Gaussian (z.z, not |z|^2);
* red-black ordering: red = even sum of node indices, red before black in
  both pre- and post-smoothing;
* the coarse operators are rediscretisations (same stencil, coarse h, chi at
  the coarse nodes, which are a subset of the fine nodes);
* the coarsest level is solved directly with a dense LU with partial pivoting.

Layout used throughout: an array of shape (m,)*d holds the (n-2)^d interior
unknowns, axis -1 is x (component 0 of eta/alpha), axis -2 is y, axis -3 is z.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

LN2 = math.log(2.0)


# ---------------------------------------------------------------------------
# Sec. 3.3: rotation-angle helpers
# ---------------------------------------------------------------------------
def gamma_from_ecs(theta: float) -> float:
    """eq. (thetagamma): rotation angle matched to an ECS layer of angle theta
    covering a quarter of the box per side."""
    return math.atan(math.sin(theta) / (2.0 + math.cos(theta)))


def min_gamma(beta_min: float = 0.5) -> float:
    """eq. (mingammajac): smallest rotation keeping Jacobi/GS multigrid stable
    for a complex shift beta_min."""
    return math.atan(beta_min) / 2.0


def csl_shift(gamma: float) -> complex:
    """eq. (csl): multiplying eq. (csg) by e^{i phi}, phi = 2 gamma, turns the
    rotated grid into a complex-shifted Laplacian with shift alpha + i beta."""
    return complex(math.cos(2 * gamma), math.sin(2 * gamma))


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------
@dataclass
class Gaussian:
    """One term A exp(-sum_c (z_c - center_c)^2 / w) of the potential chi."""
    amp: complex
    width: float
    center: tuple = (0.0, 0.0, 0.0)


@dataclass
class Problem:
    dim: int
    n: int                      # nodes per dimension, 2^L + 1
    lo: float
    hi: float
    gamma: float                # rotation angle of the contour (radians)
    k: float                    # wavenumber k_0
    gaussians: list = field(default_factory=list)

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / (self.n - 1)

    @property
    def m(self) -> int:
        return self.n - 2


def interior_coords(n: int, lo: float, hi: float) -> np.ndarray:
    """Real coordinates x_i = lo + i h of the interior nodes i = 1..n-2."""
    h = (hi - lo) / (n - 1)
    return lo + h * np.arange(1, n - 1, dtype=np.float64)


def _axis_coords(dim: int, n: int, lo: float, hi: float):
    """Per-component coordinate arrays broadcastable to the (m,)*d layout.
    Component c (x=0, y=1, z=2) varies along array axis dim-1-c."""
    x = interior_coords(n, lo, hi)
    out = []
    for c in range(dim):
        shape = [1] * dim
        shape[dim - 1 - c] = x.size
        out.append(x.reshape(shape))
    return out


def chi_at_nodes(prob: Problem, n: int | None = None) -> np.ndarray:
    """chi evaluated at the complex nodes z = x e^{i gamma} (Sec. 3.1, analytic
    continuation of the real potential) on the grid with n nodes per side."""
    n = prob.n if n is None else n
    rot = np.exp(1j * prob.gamma)
    X = _axis_coords(prob.dim, n, prob.lo, prob.hi)
    chi = np.zeros((n - 2,) * prob.dim, dtype=np.complex128)
    for g in prob.gaussians:
        s = 0.0
        for c in range(prob.dim):
            zc = rot * X[c]
            s = s + (zc - g.center[c]) ** 2
        chi = chi + complex(g.amp) * np.exp(-s / g.width)
    return chi


def u_incident(prob: Problem, eta, n: int | None = None) -> np.ndarray:
    """u_in(z) = exp(i k eta.z) at the complex nodes (Sec. 2.1)."""
    n = prob.n if n is None else n
    rot = np.exp(1j * prob.gamma)
    X = _axis_coords(prob.dim, n, prob.lo, prob.hi)
    ph = 0.0
    for c in range(prob.dim):
        ph = ph + eta[c] * X[c]
    return np.exp(1j * prob.k * rot * ph) * np.ones((n - 2,) * prob.dim)


def chi_u_incident(prob: Problem, eta, n: int | None = None) -> np.ndarray:
    """chi(z) u_in(z) = sum_g A_g exp(-sum_c (z_c - c_c)^2 / w_g + i k eta.z),
    each term one exponential of its summed exponent: the factors alone can
    exceed the FP64 range (|u_in| = e^{k sin(gamma) |eta.x|}) where the product
    does not."""
    n = prob.n if n is None else n
    rot = np.exp(1j * prob.gamma)
    X = _axis_coords(prob.dim, n, prob.lo, prob.hi)
    ph = 0.0
    for c in range(prob.dim):
        ph = ph + eta[c] * X[c]
    out = np.zeros((n - 2,) * prob.dim, dtype=np.complex128)
    for g in prob.gaussians:
        s = 0.0
        for c in range(prob.dim):
            s = s + (rot * X[c] - g.center[c]) ** 2
        out = out + complex(g.amp) * np.exp(-s / g.width + 1j * prob.k * rot * ph)
    return out


def rhs(prob: Problem, eta) -> np.ndarray:
    """b = k^2 chi(z) u_in(z), the source of eq. (helmholtz_cc)."""
    return prob.k ** 2 * chi_u_incident(prob, eta)


# ---------------------------------------------------------------------------
# Multigrid hierarchy (Sec. 4): rediscretised operators on nested grids
# ---------------------------------------------------------------------------
@dataclass
class Level:
    dim: int
    n: int
    h: float
    c: complex                  # e^{-2i gamma} / h^2
    q: np.ndarray               # k^2 (1 + chi) at the interior nodes
    diag: np.ndarray            # 2d c - q, the diagonal of A

    @property
    def m(self) -> int:
        return self.n - 2


def make_level(prob: Problem, n: int) -> Level:
    h = (prob.hi - prob.lo) / (n - 1)
    c = np.exp(-2j * prob.gamma) / h ** 2
    q = prob.k ** 2 * (1.0 + chi_at_nodes(prob, n))
    return Level(prob.dim, n, h, c, q, 2 * prob.dim * c - q)


def make_hierarchy(prob: Problem, coarsest_n: int) -> list:
    """Levels n, (n+1)/2, ... down to coarsest_n nodes per side."""
    levels = []
    n = prob.n
    while True:
        levels.append(make_level(prob, n))
        if n == coarsest_n:
            break
        if n < coarsest_n or (n - 1) % 2:
            raise ValueError("n must be 2^j (coarsest_n - 1) + 1")
        n = (n + 1) // 2
    return levels


def neighbour_sum(u: np.ndarray) -> np.ndarray:
    """Sum of the 2d axis neighbours, zero outside the interior (Dirichlet ring)."""
    d = u.ndim
    up = np.pad(u, 1)
    s = np.zeros_like(u)
    for ax in range(d):
        lo = [slice(1, -1)] * d
        hi = [slice(1, -1)] * d
        lo[ax] = slice(0, -2)
        hi[ax] = slice(2, None)
        s = s + up[tuple(lo)] + up[tuple(hi)]
    return s


def apply_A(lv: Level, u: np.ndarray) -> np.ndarray:
    """A u = e^{-2i gamma}(2d u - sum_nbr u)/h^2 - k^2(1+chi) u  (eq. csg read
    with the Sec. 5.2 stencil)."""
    return lv.c * (2 * lv.dim * u - neighbour_sum(u)) - lv.q * u


def residual(lv: Level, u: np.ndarray, b: np.ndarray) -> np.ndarray:
    return b - apply_A(lv, u)


def assemble_matrix(lv: Level) -> sp.csr_matrix:
    """Sparse A as a sum of Kronecker products of the 1D tridiagonal
    [-1 2 -1] (the matrix L of eq. csg), scaled by e^{-2i gamma}/h^2, minus the
    diagonal k^2(1+chi).  Built independently of apply_A."""
    m = lv.m
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.identity(m)
    L = None
    for ax in range(lv.dim):
        f = [I] * lv.dim
        f[ax] = T
        term = f[0]
        for g in f[1:]:
            term = sp.kron(term, g)
        L = term if L is None else L + term
    return (lv.c * L - sp.diags(lv.q.ravel())).tocsr().astype(np.complex128)


def direct_solve(prob: Problem, b: np.ndarray) -> np.ndarray:
    """Sparse direct solve of A u = b on the finest grid (SuperLU)."""
    lv = make_level(prob, prob.n)
    A = assemble_matrix(lv).tocsc()
    return spla.spsolve(A, b.ravel()).reshape(b.shape)


# ---------------------------------------------------------------------------
# Smoothers (Sec. 4: omega-Jacobi; red-black Gauss-Seidel)
# ---------------------------------------------------------------------------
def jacobi(lv: Level, u, b, omega):
    """u <- u + omega D^{-1}(b - A u), all points from the old iterate."""
    return u + omega * residual(lv, u, b) / lv.diag


def red_mask(dim: int, m: int) -> np.ndarray:
    """True where the sum of node indices (interior index + 1 per axis) is even."""
    idx = np.indices((m,) * dim).sum(axis=0) + dim
    return (idx % 2) == 0


def rbgs(lv: Level, u, b):
    """One red-black Gauss-Seidel sweep: all red points, then all black points,
    each updated with the current values of its neighbours."""
    u = u.copy()
    red = red_mask(lv.dim, lv.m)
    for mask in (red, ~red):
        r = residual(lv, u, b)
        u[mask] = u[mask] + r[mask] / lv.diag[mask]
    return u


# ---------------------------------------------------------------------------
# Grid transfers (Sec. 4): full weighting and bi/trilinear interpolation
# ---------------------------------------------------------------------------
def restrict_fw(r: np.ndarray) -> np.ndarray:
    """Full weighting: tensor product of [1/4 1/2 1/4] centred on each coarse
    node.  Coarse interior index P sits on fine interior index 2P+1."""
    d = r.ndim
    mf = r.shape[0]
    mc = (mf - 1) // 2
    out = np.zeros((mc,) * d, dtype=r.dtype)
    for off in np.ndindex(*(3,) * d):
        w = 1.0
        sl = []
        for o in off:
            w *= 0.5 if o == 1 else 0.25
            sl.append(slice(o, o + 2 * mc, 2))
        out = out + w * r[tuple(sl)]
    return out


def _interp_axis(E: np.ndarray, ax: int) -> np.ndarray:
    """Linear interpolation of node values (boundary included) along one axis:
    fine node 2I takes E[I], fine node 2I+1 takes (E[I] + E[I+1]) / 2."""
    nc = E.shape[ax]
    shape = list(E.shape)
    shape[ax] = 2 * nc - 1
    F = np.zeros(shape, dtype=E.dtype)
    even = [slice(None)] * E.ndim
    odd = [slice(None)] * E.ndim
    even[ax] = slice(0, None, 2)
    odd[ax] = slice(1, None, 2)
    a = [slice(None)] * E.ndim
    b = [slice(None)] * E.ndim
    a[ax] = slice(0, -1)
    b[ax] = slice(1, None)
    F[tuple(even)] = E
    F[tuple(odd)] = 0.5 * (E[tuple(a)] + E[tuple(b)])
    return F


def prolong(e: np.ndarray) -> np.ndarray:
    """Bi/trilinear interpolation of a coarse interior field (zero on the
    coarse boundary ring) to the fine interior."""
    E = np.pad(e, 1)
    for ax in range(e.ndim):
        E = _interp_axis(E, ax)
    return E[(slice(1, -1),) * e.ndim]


# ---------------------------------------------------------------------------
# Coarsest-level direct solve
# ---------------------------------------------------------------------------
def coarse_factor(lv: Level):
    """Dense LU with partial pivoting of the coarsest operator."""
    A = assemble_matrix(lv).toarray()
    return sla.lu_factor(A)


def coarse_solve(lu, b: np.ndarray) -> np.ndarray:
    return sla.lu_solve(lu, b.ravel()).reshape(b.shape)


# ---------------------------------------------------------------------------
# V-cycle and the iteration around it
# ---------------------------------------------------------------------------
@dataclass
class MGOptions:
    smoother: str = "jacobi"     # "jacobi", "rbgs" or "gmres"
    omega: float = 2.0 / 3.0
    nu1: int = 1
    nu2: int = 1
    coarsest_n: int = 5
    rel_tol: float = 1e-8
    max_cycles: int = 100
    krylov_m: int = 3            # GMRES(m) smoothing steps


def gmres_smooth(lv: Level, u: np.ndarray, b: np.ndarray, m: int) -> np.ndarray:
    """One GMRES(m) cycle used as a smoothing step (Sec. 3.3: a Krylov smoother
    such as GMRES(m), m = 2 or 3, replaces omega-Jacobi / Gauss-Seidel so that
    rotation angles near 10 degrees stay stable; Tables 2-3 use GMRES(3)).

    From the iterate u with r0 = b - A u and beta = ||r0||: Arnoldi with
    modified Gram-Schmidt builds an orthonormal V_{k+1} and the (k+1) x k upper
    Hessenberg H with A V_k = V_{k+1} H (k = m unless h_{j+1,j} = 0 ends it
    early); y minimises ||beta e_1 - H y||_2, and u + V_k y is returned -- the
    iterate of least residual norm in u + span{r0, A r0, ..., A^{k-1} r0}."""
    r0 = residual(lv, u, b)
    beta = norm2(r0)
    if beta == 0.0:
        return u.copy()
    V = [r0 / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    k = 0
    for j in range(m):
        w = apply_A(lv, V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = norm2(w)
        k = j + 1
        if H[j + 1, j] == 0.0:
            break
        V.append(w / H[j + 1, j])
    g = np.zeros(k + 1, dtype=np.complex128)
    g[0] = beta
    y = np.linalg.lstsq(H[:k + 1, :k], g, rcond=None)[0]
    du = np.zeros_like(u)
    for j in range(k):
        du = du + y[j] * V[j]
    return u + du


def _smooth(lv, u, b, opts):
    if opts.smoother == "jacobi":
        return jacobi(lv, u, b, opts.omega)
    if opts.smoother == "rbgs":
        return rbgs(lv, u, b)
    if opts.smoother == "gmres":
        return gmres_smooth(lv, u, b, opts.krylov_m)
    raise ValueError(opts.smoother)


def vcycle(levels, lu, l, u, b, opts):
    """One V(nu1, nu2) cycle on level l for A_l u = b (Sec. 4)."""
    lv = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(lu, b)
    for _ in range(opts.nu1):
        u = _smooth(lv, u, b, opts)
    bc = restrict_fw(residual(lv, u, b))
    ec = vcycle(levels, lu, l + 1, np.zeros_like(bc), bc, opts)
    u = u + prolong(ec)
    for _ in range(opts.nu2):
        u = _smooth(lv, u, b, opts)
    return u


def norm2(v: np.ndarray) -> float:
    """Euclidean norm with a power-of-two prescale so that squares of values
    up to the FP64 limit do not overflow."""
    a = np.abs(v)
    mx = a.max() if a.size else 0.0
    if mx == 0.0 or not np.isfinite(mx):
        return float(mx)
    s = math.ldexp(1.0, math.frexp(mx)[1] - 1)
    return float(s * np.sqrt(np.sum((a / s) ** 2)))


@dataclass
class SolveResult:
    u: np.ndarray
    history: list               # ||r_k|| / ||b||, k = 0, 1, ...
    cycles: int
    converged: bool

    @property
    def conv_factor(self) -> float:
        """Average convergence factor (||r_k||/||r_0||)^(1/k)."""
        if self.cycles == 0:
            return 0.0
        return self.history[-1] ** (1.0 / self.cycles)


def mg_solve(prob: Problem, b: np.ndarray, opts: MGOptions, u0=None) -> SolveResult:
    """Repeat V-cycles from u0 (default 0) until ||b - A u|| <= rel_tol ||b||."""
    levels = make_hierarchy(prob, opts.coarsest_n)
    lu = coarse_factor(levels[-1])
    u = np.zeros_like(b) if u0 is None else u0.copy()
    nb = norm2(b)
    if nb == 0.0:
        return SolveResult(np.zeros_like(b), [0.0], 0, True)
    hist = [norm2(residual(levels[0], u, b)) / nb]
    cycles = 0
    while hist[-1] > opts.rel_tol and cycles < opts.max_cycles:
        u = vcycle(levels, lu, 0, u, b, opts)
        cycles += 1
        hist.append(norm2(residual(levels[0], u, b)) / nb)
        if not np.isfinite(hist[-1]):
            break
    return SolveResult(u, hist, cycles, hist[-1] <= opts.rel_tol)


@dataclass
class FMGResult:
    u: np.ndarray
    level_cycles: list          # V-cycles on each level above the coarsest, coarse to fine
    level_history: list         # per level: ||r_k|| / ||b_l||, k = 0 (interpolated guess), 1, ...
    converged: bool

    @property
    def cycles(self) -> int:
        """V-cycles on the finest level."""
        return self.level_cycles[-1] if self.level_cycles else 0

    @property
    def history(self) -> list:
        return self.level_history[-1] if self.level_history else [0.0]


def fmg_solve(prob: Problem, b: np.ndarray, opts: MGOptions) -> FMGResult:
    """Full multigrid (Sec. 4, the FMG paragraph with Table 3): a nested
    iteration of V-cycles.  The right-hand side is carried to every coarser
    level by full weighting, b_{l+1} = FW(b_l); the coarsest level is solved
    directly; then on each finer level, from the second coarsest up to the
    finest, the bi/trilinear interpolation of the coarser level's solution is
    the initial guess of V(nu1, nu2)-cycles on A_l u_l = b_l, run until
    ||b_l - A_l u_l|| <= rel_tol ||b_l|| (the same tolerance on every level)
    or max_cycles.  The paper does not say how the coarse right-hand sides are
    formed or what the tolerance is relative to; these are the readings taken."""
    levels = make_hierarchy(prob, opts.coarsest_n)
    lu = coarse_factor(levels[-1])
    bs = [b]
    for _ in levels[1:]:
        bs.append(restrict_fw(bs[-1]))
    u = coarse_solve(lu, bs[-1])
    counts, hists = [], []
    converged = True
    for l in range(len(levels) - 2, -1, -1):
        u = prolong(u)
        lv = levels[l]
        nb = norm2(bs[l])
        hist = [norm2(residual(lv, u, bs[l])) / nb] if nb > 0 else [0.0]
        c = 0
        while hist[-1] > opts.rel_tol and c < opts.max_cycles:
            u = vcycle(levels[l:], lu, 0, u, bs[l], opts)
            c += 1
            hist.append(norm2(residual(lv, u, bs[l])) / nb)
            if not np.isfinite(hist[-1]):
                break
        counts.append(c)
        hists.append(hist)
        converged = converged and hist[-1] <= opts.rel_tol
    return FMGResult(u, counts, hists, converged)


# ---------------------------------------------------------------------------
# Far field (eq. FFmap over the contour, eq. I2complex)
# ---------------------------------------------------------------------------
def far_field(prob: Problem, u: np.ndarray, eta, alphas, return_terms_norm=False):
    """F(alpha) = k^2 e^{i d gamma} h^d sum_j e^{-i k z_j.alpha} chi_j (u_in,j + u_j).

    Returns (mant, e2[, tnorm]) with F = mant * 2**e2 so that results beyond the
    FP64 range stay representable.  The per-angle exponent is the exponent of
    the largest term, found exactly; every term is formed from its logarithm,
    so nothing overflows.  tnorm = sum_j |term_j| * 2**-e2 (condition number
    kappa = tnorm / |mant|)."""
    alphas = np.atleast_2d(np.asarray(alphas, dtype=np.float64))
    rot = np.exp(1j * prob.gamma)
    X = _axis_coords(prob.dim, prob.n, prob.lo, prob.hi)
    g = chi_u_incident(prob, eta) + chi_at_nodes(prob) * u
    with np.errstate(divide="ignore"):
        lg = np.log(np.abs(g))
    ag = np.angle(g)
    pref = prob.k ** 2 * np.exp(1j * prob.dim * prob.gamma) * prob.h ** prob.dim
    mant = np.zeros(len(alphas), dtype=np.complex128)
    e2 = np.zeros(len(alphas), dtype=np.int64)
    tn = np.zeros(len(alphas), dtype=np.float64)
    for a, al in enumerate(alphas):
        ax = 0.0
        for c in range(prob.dim):
            ax = ax + al[c] * X[c]
        ph = -1j * prob.k * rot * ax          # log of e^{-i k z.alpha}
        logmag = ph.real + lg                 # log |term_j| (before the prefactor)
        top = np.max(logmag)
        if not np.isfinite(top):
            continue
        s = math.floor(top / LN2)
        terms = np.exp(logmag - s * LN2 + 1j * (ph.imag + ag))
        mant[a] = pref * np.sum(terms)
        e2[a] = s
        tn[a] = abs(pref) * np.sum(np.abs(terms))
    if return_terms_norm:
        return mant, e2, tn
    return mant, e2


def far_field_value(mant, e2):
    """F = mant * 2**e2 as complex128 (inf where it does not fit)."""
    with np.errstate(over="ignore", invalid="ignore"):
        sc = np.array([math.ldexp(1.0, int(min(e, 2000))) if e < 1024 else np.inf for e in np.atleast_1d(e2)])
        return np.atleast_1d(mant) * sc


def born_far_field(k: float, amp: complex, width: float, dim: int, eta, alpha) -> complex:
    """First Born approximation for chi = A exp(-|x|^2/w): the Fourier integral
    k^2 A int exp(-|x|^2/w + i k (eta - alpha).x) dx in closed form."""
    q2 = float(np.sum((np.asarray(eta, float) - np.asarray(alpha, float)) ** 2))
    return k ** 2 * amp * (math.pi * width) ** (dim / 2.0) * math.exp(-width * k ** 2 * q2 / 4.0)


# ---------------------------------------------------------------------------
# Angle sets used by the model problems
# ---------------------------------------------------------------------------
def angles_2d(n_ang: int) -> np.ndarray:
    t = 2 * np.pi * np.arange(n_ang) / n_ang
    return np.stack([np.cos(t), np.sin(t)], axis=1)


def angles_3d(n_phi: int, n_theta: int) -> np.ndarray:
    """phi_i = 2 pi i / n_phi, theta_j = pi (j + 1/2) / n_theta; row a = j*n_phi + i."""
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    th = np.pi * (np.arange(n_theta) + 0.5) / n_theta
    out = []
    for t in th:
        for p in ph:
            out.append([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])
    return np.array(out)


# ---------------------------------------------------------------------------
# Plain-dict marshalling (the shared input generators describe problems as dicts)
# ---------------------------------------------------------------------------
def problem_from_dict(p: dict) -> Problem:
    gs = [Gaussian(complex(g["amp"]), float(g["width"]), tuple(g.get("center", (0.0, 0.0, 0.0))))
          for g in p["gaussians"]]
    return Problem(int(p["dim"]), int(p["n"]), float(p["lo"]), float(p["hi"]), float(p["gamma"]),
                   float(p["k"]), gs)


def opts_from_dict(o: dict) -> MGOptions:
    return MGOptions(smoother=o.get("smoother", "jacobi"), omega=float(o.get("omega", 2.0 / 3.0)),
                     nu1=int(o.get("nu1", 1)), nu2=int(o.get("nu2", 1)),
                     coarsest_n=int(o.get("coarsest_n", 5)), rel_tol=float(o.get("rel_tol", 1e-8)),
                     max_cycles=int(o.get("max_cycles", 100)), krylov_m=int(o.get("krylov_m", 3)))
