"""Plain FP64 CPU oracle for the 2D partial-wave Schroedinger problem on a
complex contour and its ionization amplitudes (Sec. 5.2-5.3).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and ``bench.py``'s CPU arm,
never by the product path; it shares no code with the CUDA library.

Model (Sec. 5.2, eq. partialwave2d with its boundary conditions):
  (-1/2 Delta + V1(x) + V2(y) + V12(x,y) - E) u = phi,   x, y >= 0,
  u = 0 on x = 0 and y = 0, outgoing for large x or y,
with V1(x) = -4.5 e^{-x^2}, V2(y) = -4.5 e^{-y^2}, V12 = 2 e^{-(x+y)^2} and
phi = e^{-3(x+y)^2}.  The complex contour (Sec. 5.3): every coordinate is
rotated, z = x e^{i gamma} on [0, R] with R = 15 and gamma about 8.5 degrees,
and u = 0 at z = 0 and z = R e^{i gamma} (the rotation damps the outgoing
waves, as on the Helmholtz contour).  Multiplied by 2 the equation is
  -Delta_z u - q u = 2 phi,   q = 2E - 2(V1 + V2 + V12),
the five-point stencil with the complex spacing h e^{i gamma}.

Amplitudes (eqs. single-ionization and double-ionization), evaluated along
the contour with the Jacobian e^{2 i gamma} and uniform weights h^2:
  s_n(E)    = int phi_{k_n}(x) phi_n(y) [phi - V12 u] dx dy,   k_n = sqrt(2 (E - lambda_n)),
  f(k1, k2) = int phi_{k1}(x) phi_{k2}(y) [phi - V12 u] dx dy,  k1 = sqrt(2E) sin a, k2 = sqrt(2E) cos a,
with phi_n the bound states of eq. (boundstate), (-1/2 d^2/dx^2 + V1) phi_n =
lambda_n phi_n, phi_n(0) = 0, and phi_k the regular solution of eq.
(testfunction) normalised to sin(k x + delta) / sqrt(k) where V1 has died out.

Readings (each repeated in the design notes): the bound state is normalised
by int phi_n(z)^2 dz = 1 along the contour (the analytic continuation of the
real normalisation; no complex conjugate); lambda_n enters k_n by its real
part (the contour eigenvalue is real up to discretisation error); the
asymptotic fit of phi_k uses the discrete wavenumber of the recurrence.  The
paper prints sigma(k1, k2) = 8 pi^2 / k0^2 |f|^2 / (k1 k2) but no k0 for this
model (it has no incident wave) and no formula for the single ionization cross
section; the cross sections are read as single = 4 |s_0|^2 and total double =
int_0^E (4/pi) |f|^2 d eps = (4/pi) int_0^{pi/2} |f(a)|^2 k1 k2 da
(eps = E sin^2 a, d eps = k1 k2 da), the constants set by the scale of Fig. 8;
the figure then pins the energy dependence.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

GAMMA_PW = 8.5 * math.pi / 180.0      # Sec. 5.3: overall rotation about 8.5 degrees
R_PW = 15.0                           # Sec. 5.3: numerical domain [0, 15]^2


def contour_nodes(n: int, R: float = R_PW, gamma: float = GAMMA_PW) -> np.ndarray:
    """Interior nodes z_i = i h e^{i gamma}, i = 1 .. n-2, h = R / (n - 1)."""
    h = R / (n - 1)
    return np.arange(1, n - 1) * h * np.exp(1j * gamma)


def v1(z):
    return -4.5 * np.exp(-z * z)


def v12(zx, zy):
    return 2.0 * np.exp(-(zx + zy) ** 2)


def phi_rhs(zx, zy):
    return np.exp(-3.0 * (zx + zy) ** 2)


def fields(n: int, R: float = R_PW, gamma: float = GAMMA_PW):
    """(V1(x) + V2(y) + V12, V12, phi) at the interior nodes, arrays (m, m)
    with axis -1 = x and axis -2 = y."""
    z = contour_nodes(n, R, gamma)
    ZY, ZX = np.meshgrid(z, z, indexing="ij")
    w12 = v12(ZX, ZY)
    return v1(ZX) + v1(ZY) + w12, w12, phi_rhs(ZX, ZY)


def q_of(E: float, n: int, R: float = R_PW, gamma: float = GAMMA_PW) -> np.ndarray:
    """q = 2E - 2(V1 + V2 + V12): the operator is A u = c (4 u - sum_nbr u) - q u
    with c = e^{-2 i gamma} / h^2."""
    V, _, _ = fields(n, R, gamma)
    return 2.0 * E - 2.0 * V


def assemble(E: float, n: int, R: float = R_PW, gamma: float = GAMMA_PW) -> sp.csr_matrix:
    """Sparse A = -Delta_z - q (Dirichlet at both ends of both contours)."""
    m = n - 2
    h = R / (n - 1)
    c = np.exp(-2j * gamma) / h ** 2
    T = sp.diags([-np.ones(m - 1), 2.0 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1], format="csr")
    I = sp.identity(m, format="csr")
    L = sp.kron(I, T) + sp.kron(T, I)
    return (c * L - sp.diags(q_of(E, n, R, gamma).ravel())).tocsr()


def solve(E: float, n: int, R: float = R_PW, gamma: float = GAMMA_PW) -> np.ndarray:
    """u of (H - E) u = phi along the contour by a sparse direct solve."""
    _, _, ph = fields(n, R, gamma)
    A = assemble(E, n, R, gamma)
    m = n - 2
    return spla.spsolve(A.tocsc(), 2.0 * ph.ravel()).reshape(m, m)


# ---------------------------------------------------------------------------
# 1D functions along the contour (eqs. boundstate and testfunction)
# ---------------------------------------------------------------------------
def hamiltonian_1d(n: int, R: float = R_PW, gamma: float = GAMMA_PW) -> np.ndarray:
    """Dense H1 = -1/2 d^2/dz^2 + V1(z) on the interior nodes (Dirichlet)."""
    m = n - 2
    hz = R / (n - 1) * np.exp(1j * gamma)
    z = contour_nodes(n, R, gamma)
    H = np.diag(1.0 / hz ** 2 + v1(z)).astype(np.complex128)
    off = -0.5 / hz ** 2
    H += np.diag(np.full(m - 1, off), 1) + np.diag(np.full(m - 1, off), -1)
    return H


def bound_states(n: int, R: float = R_PW, gamma: float = GAMMA_PW):
    """Eigenpairs of H1 with negative real part, lowest first; each phi_n
    normalised by sum_i phi_n(z_i)^2 h e^{i gamma} = 1 and phase-fixed so that
    its largest entry is real positive."""
    H = hamiltonian_1d(n, R, gamma)
    lam, vec = sla.eig(H)
    idx = [i for i in np.argsort(lam.real) if lam[i].real < 0.0]
    hz = R / (n - 1) * np.exp(1j * gamma)
    out = []
    for i in idx:
        v = vec[:, i]
        v = v / np.sqrt(np.sum(v * v) * hz)
        j = np.argmax(np.abs(v))
        if v[j].real < 0:
            v = -v
        out.append((lam[i], v))
    return out


def regular_solution(k: float, n: int, R: float = R_PW, gamma: float = GAMMA_PW, tail: float = 1e-15, pot=v1):
    """Regular solution of (-1/2 d^2 + V1 - k^2/2) phi = 0 with phi(0) = 0,
    by the three-term recurrence of the discrete equation from phi_0 = 0,
    phi_1 = h e^{i gamma}; normalised so that phi = sin(kappa z + delta)/sqrt(k)
    where |V1| < tail, kappa the discrete wavenumber (cos(kappa h_z) =
    1 - (k h_z)^2 / 2).  Returns phi at the interior nodes."""
    m = n - 2
    hz = R / (n - 1) * np.exp(1j * gamma)
    z = np.concatenate([[0.0], contour_nodes(n, R, gamma)])
    p = np.zeros(m + 1, dtype=np.complex128)
    p[1] = hz
    vz = pot(z) + 0j * z
    w = 2.0 * hz * hz * (vz - 0.5 * k * k)
    for i in range(1, m):
        p[i + 1] = 2.0 * p[i] - p[i - 1] + w[i] * p[i]
    theta = np.arccos(1.0 - 0.5 * (k * hz) ** 2 + 0j)
    if theta.imag < 0:
        theta = -theta
    far = np.nonzero(np.abs(vz) < tail)[0]
    i0 = int(far[0])
    M = np.array([[np.exp(1j * theta * i0), np.exp(-1j * theta * i0)],
                  [np.exp(1j * theta * (i0 + 1)), np.exp(-1j * theta * (i0 + 1))]])
    a, b = np.linalg.solve(M, p[i0:i0 + 2])
    amp = 2.0 * np.sqrt(a * b)               # p = amp sin(theta i + delta) there
    return p[1:] / (amp * math.sqrt(k))


# ---------------------------------------------------------------------------
# Amplitudes and cross sections
# ---------------------------------------------------------------------------
def integrand(u: np.ndarray, n: int, R: float = R_PW, gamma: float = GAMMA_PW) -> np.ndarray:
    """phi - V12 u at the interior nodes."""
    _, w12, ph = fields(n, R, gamma)
    return ph - w12 * u


def contract(X: np.ndarray, Y: np.ndarray, g: np.ndarray, n: int, R: float = R_PW,
             gamma: float = GAMMA_PW) -> np.ndarray:
    """out[r] = e^{2 i gamma} h^2 sum_{j,i} X[r, i] Y[r, j] g[j, i] (x index i,
    y index j): the contour quadrature of int X_r(x) Y_r(y) g(x, y)."""
    h = R / (n - 1)
    return np.exp(2j * gamma) * h * h * np.einsum("ri,rj,ji->r", X, Y, g)


def single_amplitude(E: float, u: np.ndarray, n: int, R: float = R_PW, gamma: float = GAMMA_PW, state: int = 0):
    lam, ph_n = bound_states(n, R, gamma)[state]
    kn = math.sqrt(2.0 * (E - lam.real))
    X = regular_solution(kn, n, R, gamma)[None, :]
    return contract(X, ph_n[None, :], integrand(u, n, R, gamma), n, R, gamma)[0], kn


def double_amplitudes(E: float, u: np.ndarray, alphas: np.ndarray, n: int, R: float = R_PW,
                      gamma: float = GAMMA_PW) -> np.ndarray:
    k = math.sqrt(2.0 * E)
    X = np.stack([regular_solution(k * math.sin(a), n, R, gamma) for a in alphas])
    Y = np.stack([regular_solution(k * math.cos(a), n, R, gamma) for a in alphas])
    return contract(X, Y, integrand(u, n, R, gamma), n, R, gamma)


def alpha_midpoints(n_alpha: int) -> np.ndarray:
    """Midpoint nodes a_j = (j + 1/2) pi / (2 n_alpha) of [0, pi/2]."""
    return (np.arange(n_alpha) + 0.5) * (math.pi / 2) / n_alpha


def double_cross_section(f: np.ndarray, alphas: np.ndarray, E: float) -> float:
    """Total double ionization cross section int_0^E sigma d eps with
    eps = E sin^2 a (d eps = k1 k2 da), read as (4/pi) int_0^{pi/2} |f(a)|^2 k1 k2 da
    (midpoint rule over the given midpoint nodes)."""
    k = math.sqrt(2.0 * E)
    k1k2 = k * k * np.sin(alphas) * np.cos(alphas)
    return (4.0 / math.pi) * float(np.sum(np.abs(f) ** 2 * k1k2)) * (math.pi / 2) / len(alphas)


def single_cross_section(s: complex) -> float:
    """Single ionization cross section of the lowest bound-state channel, read
    as 4 |s_0|^2 (both channels of the x <-> y symmetric model)."""
    return 4.0 * abs(s) ** 2


# ---------------------------------------------------------------------------
# Multigrid on the contour: the levels of csff_oracle with q at each level's
# nodes (coarse nodes are fine nodes, so this is injection of q)
# ---------------------------------------------------------------------------
def mg_levels(E: float, n: int, coarsest_n: int = 5, R: float = R_PW, gamma: float = GAMMA_PW) -> list:
    from oracle import csff_oracle as O
    out = []
    while True:
        h = R / (n - 1)
        c = np.exp(-2j * gamma) / h ** 2
        q = q_of(E, n, R, gamma)
        out.append(O.Level(2, n, h, c, q, 4 * c - q))
        if n == coarsest_n:
            return out
        n = (n + 1) // 2


def mg_solve(E: float, n: int, opts, R: float = R_PW, gamma: float = GAMMA_PW, u0=None):
    """V-cycles (csff_oracle.vcycle) on A u = 2 phi until the relative residual
    meets opts.rel_tol; returns csff_oracle.SolveResult."""
    from oracle import csff_oracle as O
    lv = mg_levels(E, n, opts.coarsest_n, R, gamma)
    lu = O.coarse_factor(lv[-1])
    b = 2.0 * fields(n, R, gamma)[2]
    u = np.zeros_like(b) if u0 is None else u0.copy()
    nb = O.norm2(b)
    hist = [O.norm2(O.residual(lv[0], u, b)) / nb]
    cycles = 0
    while hist[-1] > opts.rel_tol and cycles < opts.max_cycles:
        u = O.vcycle(lv, lu, 0, u, b, opts)
        cycles += 1
        hist.append(O.norm2(O.residual(lv[0], u, b)) / nb)
        if not np.isfinite(hist[-1]):
            break
    return O.SolveResult(u, hist, cycles, hist[-1] <= opts.rel_tol)
