"""csff: complex-contour multigrid far-field maps on GB300 (sm_103a CUDA).

Thin ctypes binding over libcsff.so (declared in include/csff.h).  Every step
of the method runs in the library's CUDA kernels; this module only marshals
arguments (torch tensors -> device pointers, dicts -> C structs).  There is no
CPU fallback: importing the package fails if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcsff.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libcsff.so not found at {LIB_PATH}; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a). "
        "There is no CPU fallback.")
_lib = C.CDLL(LIB_PATH)

OK = 0
ERR_INVALID_ARG = 1
ERR_CUDA = 2
ERR_OOM = 3
ERR_NOT_CONVERGED = 4
ERR_DIVERGED = 5
ERR_NONFINITE = 6
ERR_TIMEOUT = 7
ERR_UNSUPPORTED = 8
WARN_ILL_CONDITIONED = 100

SMOOTHER = {"jacobi": 0, "rbgs": 1, "gmres": 2}
PRECISION = {"fp64": 0, "mixed": 1}
ARITH_FP64, ARITH_FP32 = 0, 1
MAX_HISTORY = 256


class Gauss(C.Structure):
    _fields_ = [("amp_re", C.c_double), ("amp_im", C.c_double), ("center", C.c_double * 3),
                ("width", C.c_double)]


class ProblemC(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int), ("box_lo", C.c_double), ("box_hi", C.c_double),
                ("gamma", C.c_double), ("k", C.c_double), ("n_gauss", C.c_int),
                ("gauss", C.POINTER(Gauss))]


class OptsC(C.Structure):
    _fields_ = [("smoother", C.c_int), ("omega", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
                ("coarsest_n", C.c_int), ("rel_tol", C.c_double), ("max_cycles", C.c_int),
                ("precision", C.c_int), ("inner_cycles", C.c_int), ("krylov_m", C.c_int),
                ("adaptive_inner", C.c_int), ("refine_fp64", C.c_int)]


class InfoC(C.Structure):
    _fields_ = [("status", C.c_int), ("cycles", C.c_int), ("refinements", C.c_int),
                ("rel_res", C.c_double), ("conv_factor", C.c_double), ("n_hist", C.c_int),
                ("history", C.c_double * MAX_HISTORY), ("flags", C.c_int)]

    def as_dict(self):
        return {"status": self.status, "cycles": self.cycles, "refinements": self.refinements,
                "rel_res": self.rel_res, "conv_factor": self.conv_factor,
                "history": list(self.history[: self.n_hist]), "flags": self.flags}


class DescC(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n", C.c_int * 16), ("h", C.c_double * 16),
                ("device_bytes", C.c_size_t), ("log_rhs_max", C.c_double), ("log_ff_max", C.c_double),
                ("ill_conditioned", C.c_int), ("below_min_gamma", C.c_int)]


class ProfStatsC(C.Structure):
    _fields_ = [("launches", C.c_int), ("ms", C.c_double), ("alg_bytes", C.c_double), ("alg_flops", C.c_double)]


PROF_FF_CONTRACT, PROF_MG32, PROF_MG64, PROF_FF_OTHER, PROF_TILES32, PROF_TILES32_FINE = 1, 2, 4, 8, 16, 32
FF_FP64, FF_TC_BF16X4 = 0, 1
PROF_NAMES = ("ff_contract", "mg32", "mg64", "ff_other", "tiles32", "tiles32_fine")

_vp, _cp, _i, _d = C.c_void_p, C.c_char_p, C.c_int, C.c_double
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_SIGS = {
    "csff_plan_create": (_i, [C.POINTER(ProblemC), C.POINTER(OptsC), _vp, C.POINTER(_vp)]),
    "csff_plan_destroy": (None, [_vp]),
    "csff_plan_set_stream": (_i, [_vp, _vp]),
    "csff_plan_describe": (_i, [_vp, C.POINTER(DescC)]),
    "csff_rhs": (_i, [_vp, _i, _dp, _vp]),
    "csff_solve": (_i, [_vp, _i, _dp, _vp, _i, C.POINTER(InfoC)]),
    "csff_solve_fmg": (_i, [_vp, _i, _dp, _vp, C.POINTER(_i), C.POINTER(InfoC)]),
    "csff_far_field": (_i, [_vp, _i, _dp, _vp, _i, _dp, _vp, _vp]),
    "csff_plan_set_far_field_mode": (_i, [_vp, _i]),
    "csff_residual": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "csff_smooth": (_i, [_vp, _i, _i, _vp, _vp, _i]),
    "csff_restrict": (_i, [_vp, _i, _i, _vp, _vp]),
    "csff_prolong_add": (_i, [_vp, _i, _i, _vp, _vp]),
    "csff_coarse_solve": (_i, [_vp, _i, _vp, _vp]),
    "csff_norm2": (_i, [_vp, _i, _i, _vp, _dp]),
    "csff_vcycle": (_i, [_vp, _i, _vp, _vp]),
    "csff_gamma_from_ecs": (_d, [_d]),
    "csff_refinement_cycles": (_i, [_d, _d, _i, _d, _i]),
    "csff_status_string": (_cp, [_i]),
    "csff_last_error": (_cp, []),
    "csff_kernel_launches": (C.c_uint64, []),
    "csff_norm2_noalloc": (_i, [_i, _vp, C.c_longlong, _i, _vp, _vp]),
    "csff_batch_create": (_i, [_i, C.POINTER(ProblemC), C.POINTER(OptsC), _vp, C.POINTER(_vp)]),
    "csff_batch_destroy": (None, [_vp]),
    "csff_batch_solve": (_i, [_vp, _dp, C.POINTER(InfoC)]),
    "csff_batch_solution": (_i, [_vp, _i, C.POINTER(_vp)]),
    "csff_batch_copy_solution": (_i, [_vp, _i, _vp]),
    "csff_batch_far_field": (_i, [_vp, _dp, C.POINTER(_i), C.POINTER(_dp), C.POINTER(_vp), C.POINTER(_vp)]),
    "csff_batch_autotune": (_i, [_vp, _dp, C.POINTER(_i), C.POINTER(_i)]),
    "csff_batch_debug_barrier": (_i, [_vp, _i, C.c_longlong]),
    "csff_batch_set_tiles": (_i, [_vp, _i, _i]),
    "csff_batch_set_learned": (_i, [_vp, _vp, _d]),
    "csff_net_num_params3": (_i, []),
    "csff_net_create3": (_i, [_fp, C.POINTER(_vp)]),
    "csff_net_forward3": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _vp]),
    "csff_net_loss_grad3": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _dp, _i, _fp, _fp, _vp]),
    "csff_net_train_step3": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _dp, _i, C.c_float, _fp, _vp]),
    "csff_net_num_params": (_i, []),
    "csff_net_create": (_i, [_fp, C.POINTER(_vp)]),
    "csff_net_destroy": (None, [_vp]),
    "csff_net_set_weights": (_i, [_vp, _fp]),
    "csff_net_get_weights": (_i, [_vp, _fp]),
    "csff_net_forward": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "csff_net_forward_mma": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "csff_net_loss_grad": (_i, [_vp, _i, _i, _i, _vp, _vp, _dp, _i, _fp, _fp, _vp]),
    "csff_net_train_step": (_i, [_vp, _i, _i, _i, _vp, _vp, _dp, _i, C.c_float, _fp, _vp]),
    "csff_plan_set_learned": (_i, [_vp, _vp, _i, _d]),
    "csff_plan_set_learned_level": (_i, [_vp, _i, _vp]),
    "csff_plan_copy_coefficients": (_i, [_vp, _i, _vp, _dp]),
    "csff_prof_begin": (_i, [C.c_uint]),
    "csff_prof_end": (_i, [C.POINTER(ProfStatsC)]),
    "csff_plan_set_potential": (_i, [_vp, _vp]),
    "csff_far_field_work": (_i, [_vp, _dp]),
    "csff_solve_rhs": (_i, [_vp, _vp, _vp, _i, C.POINTER(InfoC)]),
    "csff_plan_set_schroedinger": (_i, [_vp, _d, _vp]),
    "csff_solve_schroedinger": (_i, [_vp, _vp, _vp, _i, C.POINTER(InfoC)]),
    "csff_contour_bound_state": (_i, [_i, _d, _d, _dp, _d, _dp, _dp]),
    "csff_contour_regular_solution": (_i, [_i, _d, _d, _dp, _d, _d, _dp]),
    "csff_separable_sum": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTS = tuple(_SIGS)


class CsffError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.csff_last_error().decode() or _lib.csff_status_string(status).decode()
        super().__init__(f"{where}: {_lib.csff_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(st, where, ok=(OK,)):
    if st not in ok:
        raise CsffError(st, where)
    return st


def gamma_from_ecs(theta: float) -> float:
    """eq. (thetagamma)."""
    return _lib.csff_gamma_from_ecs(theta)


def refinement_cycles(rel_before: float, rel_after: float, cycles_run: int, rel_tol: float,
                      max_cycles: int) -> int:
    """The adaptive refinement schedule's next cycle count (csff_refinement_cycles)."""
    return int(_lib.csff_refinement_cycles(rel_before, rel_after, cycles_run, rel_tol, max_cycles))


def kernel_launches() -> int:
    return int(_lib.csff_kernel_launches())


def prof_begin(mask: int) -> None:
    """Start event-timing the selected kernel families (csff_prof_begin)."""
    _check(_lib.csff_prof_begin(mask), "prof_begin")


def prof_end() -> dict:
    out = (ProfStatsC * len(PROF_NAMES))()
    _check(_lib.csff_prof_end(out), "prof_end")
    return {PROF_NAMES[i]: {"launches": out[i].launches, "ms": out[i].ms, "alg_bytes": out[i].alg_bytes,
                            "alg_flops": out[i].alg_flops} for i in range(len(PROF_NAMES))}


NOALLOC_MAX_N = 1 << 25


def norm2_noalloc(v, out, exp_scale=0, stream=None) -> None:
    """csff_norm2_noalloc: ||v||_2 into the device double `out` without any
    device allocation (fixed scratch inside the library; see include/csff.h).
    v: contiguous complex128 or complex64 CUDA tensor; out: CUDA float64
    tensor with at least one element (the result goes to its first)."""
    import torch
    if not isinstance(v, torch.Tensor) or v.dtype not in (torch.complex128, torch.complex64):
        raise TypeError("v must be a complex128 or complex64 CUDA tensor")
    _require(v, v.dtype, v.numel(), "v")
    _require(out, torch.float64, 1, "out")
    if out.device != v.device:
        raise ValueError("v and out must be on the same device")
    arith = ARITH_FP64 if v.dtype == torch.complex128 else ARITH_FP32
    _check(_lib.csff_norm2_noalloc(arith, _ptr(v), v.numel(), int(exp_scale), _ptr(out), _stream_handle(stream)),
           "norm2_noalloc")


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _require(t, dtype, numel, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
        raise ValueError(f"{name}: need contiguous {dtype} with >= {numel} elements, got {t.dtype} {tuple(t.shape)}")


def _problem_c(problem):
    gs = problem.get("gaussians", [])
    garr = (Gauss * max(1, len(gs)))()
    for i, g in enumerate(gs):
        a = complex(g["amp"])
        c = tuple(g.get("center", (0.0, 0.0, 0.0)))
        garr[i] = Gauss(a.real, a.imag, (C.c_double * 3)(*c), float(g["width"]))
    pc = ProblemC(int(problem["dim"]), int(problem["n"]), float(problem["lo"]), float(problem["hi"]),
                  float(problem["gamma"]), float(problem["k"]), len(gs), garr)
    return pc, garr


def _opts_c(o):
    return OptsC(SMOOTHER[o.get("smoother", "jacobi")], float(o.get("omega", 2.0 / 3.0)), int(o.get("nu1", 1)),
                 int(o.get("nu2", 1)), int(o.get("coarsest_n", 5)), float(o.get("rel_tol", 1e-8)),
                 int(o.get("max_cycles", 100)), PRECISION[o.get("precision", "fp64")],
                 int(o.get("inner_cycles", 3)), int(o.get("krylov_m", 0)), int(bool(o.get("adaptive_inner", 0))),
                 int(bool(o.get("refine_fp64", 0))))


class Batch:
    """Many uneven 2D problems solved together in one persistent launch
    (csff_batch_create / csff_batch_solve)."""

    def __init__(self, problems, opts: dict, stream=None):
        self._keep = [_problem_c(p) for p in problems]
        arr = (ProblemC * len(problems))(*[k[0] for k in self._keep])
        self.n = len(problems)
        self.sizes = [(int(p["n"]) - 2) ** 2 for p in problems]
        oc = _opts_c(dict(opts, precision="mixed"))
        h = C.c_void_p()
        _check(_lib.csff_batch_create(self.n, arr, C.byref(oc), _stream_handle(stream), C.byref(h)), "batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.csff_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, eta, ok=(OK,)):
        eta, ep = _dbl(eta)
        infos = (InfoC * self.n)()
        st = _lib.csff_batch_solve(self._h, ep, infos)
        _check(st, "batch_solve", ok)
        return st, [infos[i].as_dict() for i in range(self.n)]

    def solution(self, i):
        """Copy of instance i's solution (complex128 CUDA tensor of m_i^2)."""
        import torch
        out = torch.empty(self.sizes[i], dtype=torch.complex128, device="cuda")
        _check(_lib.csff_batch_copy_solution(self._h, i, _ptr(out)), "batch_copy_solution")
        return out

    def far_field(self, eta, alphas, F, F_exp=None):
        eta, ep = _dbl(eta)
        al = [np.ascontiguousarray(a, dtype=np.float64) for a in alphas]
        n_ang = (C.c_int * self.n)(*[a.shape[0] for a in al])
        aptr = (_dp * self.n)(*[a.ctypes.data_as(_dp) for a in al])
        fptr = (C.c_void_p * self.n)(*[f.data_ptr() for f in F])
        eptr = (C.c_void_p * self.n)(*[e.data_ptr() for e in F_exp]) if F_exp is not None else None
        _check(_lib.csff_batch_far_field(self._h, ep, n_ang, aptr, fptr, eptr), "batch_far_field")

    def autotune(self, eta):
        eta, ep = _dbl(eta)
        tc, per = C.c_int(), C.c_int()
        _check(_lib.csff_batch_autotune(self._h, ep, C.byref(tc), C.byref(per)), "batch_autotune")
        return tc.value, per.value

    def set_tiles(self, tc_big, ctas_per_sm=0):
        """Fix the large levels' tile size (16 or 8) and the CTAs per SM."""
        _check(_lib.csff_batch_set_tiles(self._h, int(tc_big), int(ctas_per_sm)), "batch_set_tiles")

    def set_learned(self, net, guard=0.5):
        """Attach (net) or detach (None) the learned step on every instance's
        finest level."""
        _check(_lib.csff_batch_set_learned(self._h, net._h if net is not None else None, float(guard)),
               "batch_set_learned")
        self._net = net

    def debug_barrier(self, extra_arrivals, spin_limit=0):
        _check(_lib.csff_batch_debug_barrier(self._h, int(extra_arrivals), int(spin_limit)), "batch_debug_barrier")


class Net:
    """The learned smoother's network on the GPU (csff_net_*).  Weights are a
    flat FP32 vector, (out, in, taps) per layer: 2880 values for the 2D
    network (dim=2, 3x3), 8640 for the 3D one (dim=3, 3x3x3)."""

    def __init__(self, weights, dim=2):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim = dim
        w = np.ascontiguousarray(weights, dtype=np.float32)
        if w.size != self._n_params():
            raise ValueError("need %d weights" % self._n_params())
        h = C.c_void_p()
        create = _lib.csff_net_create if dim == 2 else _lib.csff_net_create3
        _check(create(w.ctypes.data_as(_fp), C.byref(h)), "net_create")
        self._h = h

    def _n_params(self):
        return _lib.csff_net_num_params() if self.dim == 2 else _lib.csff_net_num_params3()

    def close(self):
        if getattr(self, "_h", None):
            _lib.csff_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def weights(self):
        w = np.empty(self._n_params(), np.float32)
        _check(_lib.csff_net_get_weights(self._h, w.ctypes.data_as(_fp)), "net_get_weights")
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(_lib.csff_net_set_weights(self._h, w.ctypes.data_as(_fp)), "net_set_weights")

    def forward(self, r, y, stream=None):
        """r, y: complex64 CUDA tensors of shape (B, H, W) (2D) or (B, Z, H, W) (3D)."""
        if self.dim == 2:
            B, H, W = r.shape
            _check(_lib.csff_net_forward(self._h, B, H, W, _ptr(r), _ptr(y), _stream_handle(stream)), "net_forward")
        else:
            B, Z, H, W = r.shape
            _check(_lib.csff_net_forward3(self._h, B, Z, H, W, _ptr(r), _ptr(y), _stream_handle(stream)),
                   "net_forward3")

    def forward_mma(self, r, y, stream=None):
        """The 2D forward pass over the warp-level MMA tile (the batched
        kernel's form); r, y: complex64 CUDA tensors of shape (B, H, W)."""
        B, H, W = r.shape
        _check(_lib.csff_net_forward_mma(self._h, B, H, W, _ptr(r), _ptr(y), _stream_handle(stream)),
               "net_forward_mma")

    def loss_grad(self, r, q, c, margin=4, stream=None):
        cc, cp = _dbl(np.stack([np.real(c), np.imag(c)], axis=1).ravel())
        loss = C.c_float()
        g = np.empty(self._n_params(), np.float32)
        if self.dim == 2:
            B, H, W = r.shape
            _check(_lib.csff_net_loss_grad(self._h, B, H, W, _ptr(r), _ptr(q), cp, int(margin), C.byref(loss),
                                           g.ctypes.data_as(_fp), _stream_handle(stream)), "net_loss_grad")
        else:
            B, Z, H, W = r.shape
            _check(_lib.csff_net_loss_grad3(self._h, B, Z, H, W, _ptr(r), _ptr(q), cp, int(margin), C.byref(loss),
                                            g.ctypes.data_as(_fp), _stream_handle(stream)), "net_loss_grad3")
        return loss.value, g

    def train_step(self, r, q, c, lr, margin=4, stream=None):
        cc, cp = _dbl(np.stack([np.real(c), np.imag(c)], axis=1).ravel())
        loss = C.c_float()
        if self.dim == 2:
            B, H, W = r.shape
            _check(_lib.csff_net_train_step(self._h, B, H, W, _ptr(r), _ptr(q), cp, int(margin), float(lr),
                                            C.byref(loss), _stream_handle(stream)), "net_train_step")
        else:
            B, Z, H, W = r.shape
            _check(_lib.csff_net_train_step3(self._h, B, Z, H, W, _ptr(r), _ptr(q), cp, int(margin), float(lr),
                                             C.byref(loss), _stream_handle(stream)), "net_train_step3")
        return loss.value


def contour_bound_state(v, h, gamma, lambda_guess):
    """Bound state nearest lambda_guess of -1/2 d^2/dz^2 + V along the contour
    (csff_contour_bound_state); v: complex samples V(z_i), i = 1..m.
    Returns (lambda, phi) as (complex, complex128 numpy array)."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.complex128))
    m = v.shape[0]
    lam = np.zeros(2)
    phi = np.zeros(2 * m)
    _check(_lib.csff_contour_bound_state(m, float(h), float(gamma), v.view(np.float64).ctypes.data_as(_dp),
                                         float(lambda_guess), lam.ctypes.data_as(_dp), phi.ctypes.data_as(_dp)),
           "contour_bound_state")
    return complex(lam[0], lam[1]), phi.view(np.complex128)


def contour_regular_solution(v, h, gamma, k, tail=1e-15):
    """Regular solution of (-1/2 d^2/dz^2 + V - k^2/2) phi = 0 along the contour,
    scaled to sin(kappa z + delta)/sqrt(k) (csff_contour_regular_solution)."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.complex128))
    m = v.shape[0]
    phi = np.zeros(2 * m)
    _check(_lib.csff_contour_regular_solution(m, float(h), float(gamma), v.view(np.float64).ctypes.data_as(_dp),
                                              float(k), float(tail), phi.ctypes.data_as(_dp)),
           "contour_regular_solution")
    return phi.view(np.complex128)


class Plan:
    """A multigrid + far-field plan for one problem (csff_plan_create).

    problem: {"dim", "n", "lo", "hi", "gamma", "k", "gaussians": [{"amp", "width", "center"}]}
    opts:    {"smoother" ("jacobi" | "rbgs" | "gmres"), "omega", "nu1", "nu2", "krylov_m",
              "coarsest_n", "rel_tol", "max_cycles", "precision" ("fp64" | "mixed"), "inner_cycles"}
    """

    def __init__(self, problem: dict, opts: dict, stream=None):
        gs = problem.get("gaussians", [])
        self._g = (Gauss * max(1, len(gs)))()
        for i, g in enumerate(gs):
            a = complex(g["amp"])
            c = tuple(g.get("center", (0.0, 0.0, 0.0)))
            self._g[i] = Gauss(a.real, a.imag, (C.c_double * 3)(*c), float(g["width"]))
        self.dim = int(problem["dim"])
        self.n = int(problem["n"])
        self.m = self.n - 2
        self.N = self.m ** self.dim
        pc = ProblemC(self.dim, self.n, float(problem["lo"]), float(problem["hi"]), float(problem["gamma"]),
                      float(problem["k"]), len(gs), self._g)
        o = dict(opts)
        oc = _opts_c(o)
        self._stream = stream
        h = C.c_void_p()
        _check(_lib.csff_plan_create(C.byref(pc), C.byref(oc), _stream_handle(stream), C.byref(h)), "plan_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.csff_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._stream = stream
        _check(_lib.csff_plan_set_stream(self._h, _stream_handle(stream)), "set_stream")

    def set_far_field_mode(self, mode):
        """FF_FP64 (default) or FF_TC_BF16X4 (3D z-contraction on the tensor cores)."""
        _check(_lib.csff_plan_set_far_field_mode(self._h, int(mode)), "plan_set_far_field_mode")

    def set_learned(self, net, levels=1, guard=0.5):
        """Attach (net) or detach (None) the learned step on the finest levels."""
        _check(_lib.csff_plan_set_learned(self._h, net._h if net is not None else None, int(levels), float(guard)),
               "plan_set_learned")
        self._net = net

    def set_learned_level(self, level, net):
        """Use net (None: the plan's network) for the learned step on one level."""
        _check(_lib.csff_plan_set_learned_level(self._h, int(level), net._h if net is not None else None),
               "plan_set_learned_level")
        self._level_nets = getattr(self, "_level_nets", {})
        self._level_nets[int(level)] = net

    def coefficients(self, level):
        """(q, c): FP32 q = k^2(1+chi) of a level (complex64 CUDA tensor) and c."""
        import torch
        n = self.level_size(level)
        q = torch.empty(n, dtype=torch.complex64, device="cuda")
        cbuf = (C.c_double * 2)()
        _check(_lib.csff_plan_copy_coefficients(self._h, level, _ptr(q), cbuf), "plan_copy_coefficients")
        return q, complex(cbuf[0], cbuf[1])

    def describe(self) -> dict:
        d = DescC()
        _check(_lib.csff_plan_describe(self._h, C.byref(d)), "describe")
        return {"levels": [d.n[i] for i in range(d.n_levels)], "h": [d.h[i] for i in range(d.n_levels)],
                "device_bytes": d.device_bytes, "log_rhs_max": d.log_rhs_max, "log_ff_max": d.log_ff_max,
                "ill_conditioned": bool(d.ill_conditioned), "below_min_gamma": bool(d.below_min_gamma)}

    def level_size(self, level):
        d = DescC()
        _check(_lib.csff_plan_describe(self._h, C.byref(d)), "describe")
        return (d.n[level] - 2) ** self.dim

    # ---- whole path ------------------------------------------------------
    def rhs(self, eta, b):
        import torch
        eta, ep = _dbl(eta)
        nr = eta.shape[0]
        _require(b, torch.complex128, nr * self.N, "b")
        _check(_lib.csff_rhs(self._h, nr, ep, _ptr(b)), "rhs")

    def solve(self, eta, u, use_guess=False, ok=(OK,)):
        """Solve for each incident direction (rows of eta); u: complex128 CUDA
        tensor of n_rhs * m^d.  Returns (status, [info dicts])."""
        import torch
        eta, ep = _dbl(eta)
        nr = eta.shape[0]
        _require(u, torch.complex128, nr * self.N, "u")
        infos = (InfoC * max(1, nr))()
        st = _lib.csff_solve(self._h, nr, ep, _ptr(u), int(bool(use_guess)), infos)
        _check(st, "solve", ok)
        return st, [infos[i].as_dict() for i in range(nr)]

    def solve_fmg(self, eta, u, ok=(OK,)):
        """Full multigrid (csff_solve_fmg) for each incident direction; returns
        (status, [info dicts], level cycles per right-hand side, coarsest first)."""
        import torch
        eta, ep = _dbl(eta)
        nr = eta.shape[0]
        _require(u, torch.complex128, nr * self.N, "u")
        nl = len(self.describe()["levels"])
        cyc = (_i * max(1, nr * (nl - 1)))()
        infos = (InfoC * max(1, nr))()
        st = _lib.csff_solve_fmg(self._h, nr, ep, _ptr(u), cyc, infos)
        _check(st, "solve_fmg", ok)
        return st, [infos[i].as_dict() for i in range(nr)], \
            [list(cyc[r * (nl - 1):(r + 1) * (nl - 1)]) for r in range(nr)]

    def far_field(self, eta, u, alphas, F, F_exp=None, ok=(OK, WARN_ILL_CONDITIONED)):
        import torch
        eta, ep = _dbl(eta)
        al, ap = _dbl(alphas)
        nr, na = eta.shape[0], al.shape[0]
        _require(u, torch.complex128, nr * self.N, "u")
        _require(F, torch.complex128, nr * na, "F")
        if F_exp is not None:
            _require(F_exp, torch.int32, nr * na, "F_exp")
        st = _lib.csff_far_field(self._h, nr, ep, _ptr(u), na, ap, _ptr(F), _ptr(F_exp))
        return _check(st, "far_field", ok)

    # ---- per-step calls ----------------------------------------------------
    def _arith(self, t):
        import torch
        if t.dtype == torch.complex128:
            return ARITH_FP64
        if t.dtype == torch.complex64:
            return ARITH_FP32
        raise TypeError("buffers must be complex64 or complex128")

    def residual(self, level, u, b, r):
        _check(_lib.csff_residual(self._h, level, self._arith(u), _ptr(u), _ptr(b), _ptr(r)), "residual")

    def smooth(self, level, u, b, sweeps=1):
        _check(_lib.csff_smooth(self._h, level, self._arith(u), _ptr(u), _ptr(b), sweeps), "smooth")

    def restrict(self, level, r_fine, b_coarse):
        _check(_lib.csff_restrict(self._h, level, self._arith(r_fine), _ptr(r_fine), _ptr(b_coarse)), "restrict")

    def prolong_add(self, level, e_coarse, u_fine):
        _check(_lib.csff_prolong_add(self._h, level, self._arith(u_fine), _ptr(e_coarse), _ptr(u_fine)),
               "prolong_add")

    def coarse_solve(self, b, u):
        _check(_lib.csff_coarse_solve(self._h, self._arith(u), _ptr(b), _ptr(u)), "coarse_solve")

    def norm2(self, level, v) -> float:
        out = C.c_double()
        _check(_lib.csff_norm2(self._h, level, self._arith(v), _ptr(v), C.byref(out)), "norm2")
        return out.value

    def vcycle(self, u, b):
        _check(_lib.csff_vcycle(self._h, self._arith(u), _ptr(u), _ptr(b)), "vcycle")

    def far_field_work(self) -> float:
        """Fraction of the 2D far-field contraction the last far field computed
        (csff_far_field_work; the rest was negligible and skipped)."""
        out = C.c_double()
        _check(_lib.csff_far_field_work(self._h, C.byref(out)), "far_field_work")
        return out.value

    def set_potential(self, q):
        """q: complex128 CUDA tensor of m^d samples of q (csff_plan_set_potential)."""
        import torch
        _require(q, torch.complex128, self.N, "q")
        _check(_lib.csff_plan_set_potential(self._h, _ptr(q)), "plan_set_potential")

    def set_schroedinger(self, E, V):
        """q = 2E - 2V on the device from the potential samples V (complex128
        CUDA tensor of m^d; csff_plan_set_schroedinger)."""
        import torch
        _require(V, torch.complex128, self.N, "V")
        _check(_lib.csff_plan_set_schroedinger(self._h, float(E), _ptr(V)), "plan_set_schroedinger")

    def solve_schroedinger(self, phi, u, use_guess=False, ok=(OK,)):
        """Solve the doubled Schroedinger problem A u = 2 phi (complex128 CUDA
        tensors of m^d; csff_solve_schroedinger); returns (status, info)."""
        import torch
        _require(phi, torch.complex128, self.N, "phi")
        _require(u, torch.complex128, self.N, "u")
        info = InfoC()
        st = _lib.csff_solve_schroedinger(self._h, _ptr(phi), _ptr(u), int(bool(use_guess)), C.byref(info))
        _check(st, "solve_schroedinger", ok)
        return st, info.as_dict()

    def solve_rhs(self, b, u, use_guess=False, ok=(OK,)):
        """Solve A u = b (complex128 CUDA tensors of m^d); returns (status, info)."""
        import torch
        _require(b, torch.complex128, self.N, "b")
        _require(u, torch.complex128, self.N, "u")
        info = InfoC()
        st = _lib.csff_solve_rhs(self._h, _ptr(b), _ptr(u), int(bool(use_guess)), C.byref(info))
        _check(st, "solve_rhs", ok)
        return st, info.as_dict()

    def separable_sum(self, X, Y, f, w=None, u=None, out=None):
        """out[r] = e^{2 i gamma} h^2 sum X[r,i] Y[r,j] (f - w u)[j,i] (csff_separable_sum);
        X, Y: complex128 CUDA (n_rows, m); f, w, u: complex128 CUDA m^2."""
        import torch
        n = X.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.complex128, device=X.device)
        _check(_lib.csff_separable_sum(self._h, n, _ptr(X), _ptr(Y), _ptr(f),
                                       _ptr(w) if w is not None else None, _ptr(u) if u is not None else None,
                                       _ptr(out)), "separable_sum")
        return out
