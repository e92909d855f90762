"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

Holds problem parameter sets, angle sets, incident directions and seeded
random arrays only: none of the method's arithmetic lives here, so both the
CUDA path and the CPU oracle can take their inputs from it.

The parameter sets are synthetic stand-ins shaped like the paper's model
problems (Sec. 4 and 5: Gaussian potentials on [-R, R]^d boxes, plane-wave
incidence, equispaced outgoing angles); the paper uses no external dataset.
"""
from __future__ import annotations

import math

import numpy as np

PI = math.pi


def gauss(amp, width, center=(0.0, 0.0, 0.0)):
    return {"amp": complex(amp), "width": float(width), "center": tuple(float(c) for c in center)}


def problem(dim, n, R, gamma, k, gaussians):
    return {"dim": dim, "n": n, "lo": -float(R), "hi": float(R), "gamma": float(gamma),
            "k": float(k), "gaussians": list(gaussians)}


def angle_set_2d(n_ang):
    """alpha_a = (cos t_a, sin t_a), t_a = 2 pi a / n_ang, generated so that
    mirror images t and 2 pi - t are exact (same cosine bit for bit, sines of
    opposite sign)."""
    a = np.arange(n_ang)
    mirror = a > n_ang // 2
    j = np.where(mirror, n_ang - a, a)
    t = 2 * np.pi * j / n_ang
    s = np.where(mirror, -np.sin(t), np.sin(t))
    return np.ascontiguousarray(np.stack([np.cos(t), s], axis=1))


def angle_set_3d(n_phi, n_theta):
    """phi_i = 2 pi i / n_phi, theta_j = pi (j + 1/2) / n_theta (midpoints, no
    poles); row a = j * n_phi + i."""
    i = np.arange(n_phi)
    mirror = i > n_phi // 2
    j = np.where(mirror, n_phi - i, i)
    ph = 2 * np.pi * j / n_phi                 # phi and 2 pi - phi exact mirror images
    sgn = np.where(mirror, -1.0, 1.0)
    th = np.pi * (np.arange(n_theta) + 0.5) / n_theta
    T, P = np.meshgrid(th, ph, indexing="ij")
    S = np.broadcast_to(sgn, T.shape)
    out = np.stack([np.sin(T) * np.cos(P), S * np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    return np.ascontiguousarray(out.reshape(-1, 3))


def incident_3d_16():
    """16 incident directions on the 64x32 far-field grid: phi index
    {0,16,32,48} x theta index {5,12,19,26}; closed under eta -> -eta."""
    A = angle_set_3d(64, 32)
    rows = [j * 64 + i for j in (5, 12, 19, 26) for i in (0, 16, 32, 48)]
    return np.ascontiguousarray(A[rows])


# ---------------------------------------------------------------------------
# Model-problem parameter sets
# ---------------------------------------------------------------------------
def small_2d(k=2.0, n=65):
    """2D plain FP64 case: 65x65 on [-10,10]^2, rotation pi/6, k=2,
    chi = -0.5 exp(-|x|^2/2), eta=+x, omega-Jacobi V(2,2), 5x5 coarsest grid,
    tolerance 1e-10, 360 outgoing angles."""
    return {
        "name": "2d-n65-jacobi-fp64",
        "problem": problem(2, n, 10.0, PI / 6, k, [gauss(-0.5, 2.0)]),
        "opts": {"smoother": "jacobi", "omega": 2.0 / 3.0, "nu1": 2, "nu2": 2, "coarsest_n": 5,
                 "rel_tol": 1e-10, "max_cycles": 200},
        "eta": np.array([[1.0, 0.0]]),
        "alphas": angle_set_2d(360),
    }


def mixed_2d(k, n=1025):
    """2D FP32-inner / double-float refinement case: 1025x1025 on [-20,20]^2, rotation
    pi/6, chi = -exp(-|x|^2/4), red-black GS V(1,1), 8 levels (9x9 coarsest),
    720 outgoing angles, tolerance 1e-8."""
    coarsest = (n - 1) // 128 + 1 if n >= 1025 else 9
    return {
        "name": f"2d-n{n}-k{k:g}-rbgs",
        "problem": problem(2, n, 20.0, PI / 6, k, [gauss(-1.0, 4.0)]),
        "opts": {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": coarsest,
                 "rel_tol": 1e-8, "max_cycles": 200},
        "eta": np.array([[1.0, 0.0]]),
        "alphas": angle_set_2d(720),
    }


MIXED_2D_KS = (5.0, 10.0, 20.0, 40.0)


def big_3d(n=257, n_rhs=16):
    """3D Schroedinger-type case (Helmholtz form with k^2 = 2E): 257^3 on
    [-15,15]^3, rotation pi/6, k=4, chi = -2 exp(-|x|^2/3), 7-point stencil,
    red-black GS V(1,1), 5^3 coarsest grid, 16 incident directions, 64x32 angles."""
    eta = incident_3d_16()[:n_rhs]
    return {
        "name": f"3d-n{n}-k4-rbgs",
        "problem": problem(3, n, 15.0, PI / 6, 4.0, [gauss(-2.0, 3.0)]),
        "opts": {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5,
                 "rel_tol": 1e-8, "max_cycles": 200},
        "eta": eta,
        "alphas": angle_set_3d(64, 32),
    }


def batch_2d(n_inst=64, seed=4461, sizes=(129, 257, 513, 1025)):
    """Uneven batch: n uniform over sizes, k ~ U[2,30], amplitude ~ U[-2,-0.2],
    width sigma^2 ~ U[1,6], incidence angle ~ U[0, 2 pi); NumPy PCG64, drawn in
    that order per instance.  Box [-20,20]^2, rotation pi/6, RB-GS V(1,1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_inst):
        n = int(sizes[rng.integers(0, len(sizes))])
        k = float(rng.uniform(2.0, 30.0))
        amp = float(rng.uniform(-2.0, -0.2))
        w = float(rng.uniform(1.0, 6.0))
        t = float(rng.uniform(0.0, 2 * PI))
        out.append({
            "name": f"batch{i}",
            "problem": problem(2, n, 20.0, PI / 6, k, [gauss(amp, w)]),
            "opts": {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5,
                     "rel_tol": 1e-8, "max_cycles": 200},
            "eta": np.array([[math.cos(t), math.sin(t)]]),
            "alphas": angle_set_2d(720),
        })
    return out


def paper_window(case):
    """Same case with the Gaussian width shrunk to w' = 28/k^2, which keeps the
    largest far-field term below e^14 (inside the FP64 accuracy window)."""
    c = dict(case)
    p = dict(case["problem"])
    k = p["k"]
    p["gaussians"] = [dict(g, width=28.0 / k ** 2) for g in p["gaussians"]]
    c["problem"] = p
    c["name"] = case["name"] + "-window"
    return c


def paper_2d(gamma=14.6 * PI / 180, n=257):
    """Eq. (chi2D): k0^2 chi = -1/5 (e^{-(x^2+(y-4)^2)} + e^{-(x^2+(y+4)^2)}),
    k0 = 1 on [-20,20]^2, eta = +x."""
    return {
        "name": f"paper2d-n{n}",
        "problem": problem(2, n, 20.0, gamma, 1.0,
                           [gauss(-0.2, 1.0, (0.0, 4.0, 0.0)), gauss(-0.2, 1.0, (0.0, -4.0, 0.0))]),
        "opts": {"smoother": "jacobi", "omega": 2.0 / 3.0, "nu1": 1, "nu2": 1, "coarsest_n": 5,
                 "rel_tol": 1e-6, "max_cycles": 200},
        "eta": np.array([[1.0, 0.0]]),
        "alphas": angle_set_2d(360),
    }


def paper_gmres(dim=2, k=1.0, n=129):
    """The paper's GMRES(3)-smoothed configuration (Tables 2-3): eq. (chi2D) or
    (chi3D), k0^2 chi = -1/5 (e^{-(x^2+(y-4)^2[+z^2])} + e^{-(x^2+(y+4)^2[+z^2])}),
    on [-20,20]^d, rotation 9.9 degrees (Table 1's value for the ECS angle
    pi/6), eta = +x, V(1,1) cycles with GMRES(3) smoothing, 5^d coarsest grid,
    residual reduction 1e-6."""
    amp = -0.2 / k ** 2
    return {
        "name": f"paper-gmres-{dim}d-n{n}-k{k:g}",
        "problem": problem(dim, n, 20.0, 9.9 * PI / 180, k,
                           [gauss(amp, 1.0, (0.0, 4.0, 0.0)), gauss(amp, 1.0, (0.0, -4.0, 0.0))]),
        "opts": {"smoother": "gmres", "krylov_m": 3, "nu1": 1, "nu2": 1, "coarsest_n": 5,
                 "rel_tol": 1e-6, "max_cycles": 60},
        "eta": np.array([[1.0, 0.0] if dim == 2 else [1.0, 0.0, 0.0]]),
        "alphas": angle_set_2d(360) if dim == 2 else angle_set_3d(16, 8),
    }


def partial_wave(E, n=257, R=15.0, gamma=8.5 * PI / 180):
    """Sec. 5.2-5.3 partial-wave model along the rotated contour: V1(x) =
    -4.5 e^{-x^2}, V2(y) = -4.5 e^{-y^2}, V12 = 2 e^{-(x+y)^2}, phi =
    e^{-3(x+y)^2} on [0, R]^2 (R = 15), rotation 8.5 degrees, energy E.
    Samples at the interior nodes z = i h e^{i gamma} (x fastest): the
    potential V = V1 + V2 + V12, the source phi, V12 and V1 along one axis;
    plan options for V(1,1) cycles with GMRES(3) smoothing.  The problem's
    coefficients (q = 2E - 2V, right-hand side 2 phi) are formed by whoever
    solves it, not here."""
    h = R / (n - 1)
    z = np.arange(1, n - 1) * h * np.exp(1j * gamma)
    zy, zx = np.meshgrid(z, z, indexing="ij")
    v_one = -4.5 * np.exp(-z * z)
    w12 = 2.0 * np.exp(-(zx + zy) ** 2)
    V = -4.5 * np.exp(-zx * zx) - 4.5 * np.exp(-zy * zy) + w12
    ph = np.exp(-3.0 * (zx + zy) ** 2)
    return {
        "name": f"partial-wave-n{n}-E{E:g}",
        "problem": problem(2, n, R, gamma, 1.0, []) | {"lo": 0.0, "hi": float(R)},
        "opts": {"smoother": "gmres", "krylov_m": 3, "nu1": 1, "nu2": 1, "coarsest_n": 5,
                 "rel_tol": 1e-10, "max_cycles": 200},
        "h": h, "gamma": gamma, "E": E,
        "V": V, "f": ph, "w": w12, "v1": v_one,
    }


# ---------------------------------------------------------------------------
# Seeded random arrays
# ---------------------------------------------------------------------------
def rand_complex(shape, seed, scale=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def rand_real(shape, seed, scale=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape)
