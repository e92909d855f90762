/*
 * csff.h -- complex-contour multigrid far-field maps (C ABI).
 *
 * The method (Cools, Reps & Vanroose, "An efficient multigrid calculation of
 * the Far Field map for Helmholtz and Schroedinger equations"):
 *
 *   1. Sec. 2.1, eq. (helmholtz_in) with Sec. 3.1, eq. (helmholtz_cc): the
 *      scattered wave u solves, on the rotated grid z = x e^{i gamma},
 *          -e^{-2i gamma} Lap_h u - k^2 (1 + chi(z)) u = k^2 chi(z) u_in(z),
 *      u_in(z) = exp(i k eta.z), discretised per Sec. 3.2, eq. (csg), with the
 *      stencil of Sec. 5.2 and homogeneous Dirichlet values on the box edge.
 *   2. Sec. 4: the damped system is solved by geometric multigrid V-cycles
 *      (omega-Jacobi or red-black Gauss-Seidel smoothing, full weighting,
 *      bi/trilinear interpolation, direct solve on the coarsest grid).
 *   3. eq. (FFmap) over the contour, eq. (I2complex):
 *          F(alpha) = k^2 e^{i d gamma} h^d sum_j e^{-i k z_j.alpha}
 *                     chi(z_j) (u_in(z_j) + u(z_j))
 *      over the interior nodes (uniform weights; the paper allows any rule).
 *
 * Conventions shared by every call
 *   - d = 2 or 3; n = 2^L + 1 nodes per side on [box_lo, box_hi]^d,
 *     h = (box_hi - box_lo)/(n - 1).  Unknowns are the m^d interior nodes,
 *     m = n - 2, stored x fastest: index ((iz*m + iy)*m + ix).
 *   - Complex numbers are interleaved (re, im): "c128" = 2 x double (16 B),
 *     "c64" = 2 x float (8 B).  Directions (eta, alpha) are real unit vectors
 *     stored as d doubles per row, component 0 = x.
 *   - Pointers named *_dev are device pointers (cudaMalloc'ed or any
 *     device-accessible memory) owned by the caller; pointers named *_host are
 *     ordinary host pointers.  The library never frees caller memory.
 *   - All device work is enqueued on the plan's stream (set at creation or by
 *     csff_plan_set_stream).  Calls returning results on the host
 *     (csff_solve's info, csff_norm2) synchronise that stream.
 *   - Errors are returned, never raised: no host exit, no device trap.  On any
 *     CSFF_ERR_* the contents of output buffers are unspecified; the plan stays
 *     usable unless the error is CSFF_ERR_CUDA from a sticky CUDA fault.
 *     csff_last_error() gives a one-line description of the last failure in
 *     the calling thread.
 *   - A plan is not thread-safe; distinct plans are independent.
 *   - chi must be analytic for the contour rotation to be valid (Sec. 2.3,
 *     Sec. 3.1); the library takes chi as a sum of Gaussians and cannot check
 *     analyticity of anything else (coefficients given as samples through
 *     csff_plan_set_potential are the caller's responsibility).
 */
#ifndef CSFF_H
#define CSFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum csff_status {
  CSFF_OK = 0,
  CSFF_ERR_INVALID_ARG = 1,   /* bad pointer, size, level or option */
  CSFF_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  CSFF_ERR_OOM = 3,           /* device allocation failed */
  CSFF_ERR_NOT_CONVERGED = 4, /* max_cycles reached above rel_tol */
  CSFF_ERR_DIVERGED = 5,      /* residual grew for 3 cycles in a row */
  CSFF_ERR_NONFINITE = 6,     /* a residual norm or input became Inf/NaN */
  CSFF_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
  CSFF_ERR_UNSUPPORTED = 8,   /* option combination not built */
  CSFF_WARN_ILL_CONDITIONED = 100 /* result valid; far-field terms exceed
                                     the FP64 range or kappa is large */
} csff_status;

/* One term A exp(-sum_c (z_c - center_c)^2 / width) of chi, A = amp_re + i amp_im.
   Evaluated at complex z (analytic continuation, Sec. 3.1). */
typedef struct csff_gauss {
  double amp_re, amp_im;
  double center[3];
  double width;
} csff_gauss;

typedef struct csff_problem {
  int dim;                 /* 2 or 3 */
  int n;                   /* nodes per side, 2^L + 1, L >= 2 */
  double box_lo, box_hi;   /* box [box_lo, box_hi]^dim */
  double gamma;            /* rotation angle of the contour, radians, (0, pi/4) */
  double k;                /* wavenumber k_0 > 0 */
  int n_gauss;             /* 0..8 terms of chi */
  const csff_gauss* gauss; /* host array of n_gauss terms (copied) */
} csff_problem;

/* Smoothers (Sec. 4; GMRES(m) cycles: Sec. 3.3, Tables 2-3, for rotation
   angles near 10 degrees where the stationary smoothers diverge). */
enum { CSFF_SMOOTHER_JACOBI = 0, CSFF_SMOOTHER_RBGS = 1, CSFF_SMOOTHER_GMRES = 2 };
enum { CSFF_PREC_FP64 = 0, CSFF_PREC_MIXED = 1 };
/* Arithmetic of the per-step calls below. */
enum { CSFF_ARITH_FP64 = 0, CSFF_ARITH_FP32 = 1 };

typedef struct csff_opts {
  int smoother;       /* CSFF_SMOOTHER_* (Sec. 4) */
  double omega;       /* Jacobi weight (2/3 in the paper); ignored by RBGS */
  int nu1, nu2;       /* pre/post sweeps of V(nu1, nu2) */
  int coarsest_n;     /* nodes per side of the coarsest grid (direct solve) */
  double rel_tol;     /* stop when ||b - A u||_2 <= rel_tol ||b||_2 */
  int max_cycles;     /* FP64: V-cycles; MIXED: total FP32 V-cycles */
  int precision;      /* CSFF_PREC_FP64 or CSFF_PREC_MIXED */
  int inner_cycles;   /* MIXED: FP32 V-cycles per refinement step (>= 1; the
                         most per step with adaptive_inner) */
  int krylov_m;       /* GMRES smoother: Krylov dimension m of each GMRES(m)
                         smoothing step, 1..4 (0 selects 3); nu1 / nu2 count
                         GMRES(m) steps.  Ignored by the other smoothers. */
  int adaptive_inner; /* MIXED: 1 = after each refinement step, the next runs
                         only the FP32 cycles that the step's per-cycle
                         reduction factor predicts are needed to reach rel_tol
                         (at most inner_cycles); 0 = always inner_cycles.  Same
                         stopping test either way.  A learned smoother's
                         fallback then compares factors per inner_cycles
                         cycles. */
  int refine_fp64;    /* MIXED: 0 = the outer residual and update in double-float
                         (pairs of FP32 words, about 48 bits, on the FP32 pipes);
                         1 = in FP64 (r = b - A u, 2^-e r rounded to FP32 for the
                         cycles, u += 2^e e), as in the classical mixed-precision
                         refinement.  Both meet the same stopping test. */
} csff_opts;

#define CSFF_MAX_HISTORY 256

/* Per-solve report.  history[i] = ||r_i|| / ||b|| after i finest-level
   V-cycles (FP64) or i refinement steps (MIXED); history[0] = 1 for u0 = 0. */
typedef struct csff_info {
  int status;          /* csff_status of this right-hand side */
  int cycles;          /* finest-level V-cycles run (FP64 or FP32) */
  int refinements;     /* refinement steps (MIXED), else 0 */
  double rel_res;      /* final ||r|| / ||b|| */
  double conv_factor;  /* (||r_k|| / ||r_0||)^(1/k) per V-cycle */
  int n_hist;
  double history[CSFF_MAX_HISTORY];
  int flags;           /* bit 0: a learned smoother was attached; bit 1: it fell
                          back to plain red-black sweeps during this solve */
} csff_info;

/* Read-only description of a plan's hierarchy. */
typedef struct csff_plan_desc {
  int n_levels;
  int n[16];                 /* nodes per side of each level, finest first */
  double h[16];
  size_t device_bytes;       /* device memory held by the plan */
  double log_rhs_max;        /* estimate of max log|chi u_in| over the box */
  double log_ff_max;         /* estimate of max log|e^{-ikz.a} chi u_in| */
  int ill_conditioned;       /* 1 if log_ff_max > 600 (beyond FP64 head-room) */
  int below_min_gamma;       /* 1 if gamma < atan(0.5)/2, eq. (mingammajac) */
} csff_plan_desc;

typedef struct csff_plan csff_plan;

/* ---- plan ------------------------------------------------------------ */

/* Build the level hierarchy n, (n+1)/2, ..., coarsest_n; per level the
   complex coefficients k^2(1 + chi) and 1/diag (FP64 and FP32 copies), the
   dense inverse of the coarsest operator (FP64, from an LU with partial
   pivoting), and work buffers.  stream: a cudaStream_t (NULL = legacy
   default stream).  Sec. 3.2 eq. (csg); Sec. 4.
   Errors: CSFF_ERR_INVALID_ARG for n != 2^j (coarsest_n - 1) + 1, dim not 2/3,
   gamma outside (0, pi/4), k <= 0, n_gauss outside 0..8, bad opts;
   CSFF_ERR_OOM; CSFF_ERR_CUDA. */
csff_status csff_plan_create(const csff_problem* prob, const csff_opts* opts, void* stream,
                             csff_plan** out);
void csff_plan_destroy(csff_plan* plan);
csff_status csff_plan_set_stream(csff_plan* plan, void* stream);
csff_status csff_plan_describe(const csff_plan* plan, csff_plan_desc* desc);

/* ---- whole-path calls ------------------------------------------------ */

/* b_dev (c128, n_rhs x m^d) = k^2 chi(z) u_in(z) for each incident direction
   eta_host[r*dim ...] (Sec. 2.1). */
csff_status csff_rhs(csff_plan* plan, int n_rhs, const double* eta_host, void* b_dev);

/* Solve for the scattered wave of each incident direction.  u_dev (c128,
   n_rhs x m^d) is read as the initial guess if use_guess != 0, else taken as 0,
   and overwritten with the solution.  info_host: n_rhs reports or NULL.
   Returns the worst status over the right-hand sides (CSFF_OK if all met
   rel_tol).  FP64: V-cycles in FP64.  MIXED: iterative refinement with u, b
   and the coefficients scaled by 2^-e (e the exponent of max |b|) and held as
   double-float pairs (two FP32 words, about 48 bits): the residual
   r = b - A u formed in double-float, FP32 V-cycles on the correction
   equation A e = r, the update u += e in double-float; u is assembled in FP64
   at the end.  The coarsest-grid inverse is formed in FP64 in both; FP32
   cycles apply its FP32 rounding in FP32, since their coarse solution is
   stored in FP32 (an FP64 product would be rounded anyway). */
csff_status csff_solve(csff_plan* plan, int n_rhs, const double* eta_host, void* u_dev,
                       int use_guess, csff_info* info_host);

/* Full multigrid (Sec. 4, the FMG paragraph, and Table 3): for each incident
   direction, b = k^2 chi u_in is carried to every coarser level by full
   weighting, the coarsest level is solved directly, and on each finer level
   the bi/trilinear interpolation of the coarser solution starts V(nu1, nu2)
   cycles run until ||b_l - A_l u_l|| <= rel_tol ||b_l|| (the same tolerance
   on every level, at most max_cycles per level).  u_dev (c128, n_rhs x m^d)
   receives the finest level's iterate.  level_cycles (host, n_rhs x
   (n_levels - 1) ints, or NULL) receives the V-cycles run on each level above
   the coarsest, coarsest first; info_host (n_rhs reports or NULL) the finest
   level's: history[0] is the relative residual of the interpolated guess.
   FP64 plans only (CSFF_ERR_UNSUPPORTED otherwise).  Returns the worst status
   over the levels and right-hand sides. */
csff_status csff_solve_fmg(csff_plan* plan, int n_rhs, const double* eta_host, void* u_dev, int* level_cycles,
                           csff_info* info_host);

/* Far-field map, eq. (FFmap) over the contour (eq. I2complex), for each
   right-hand side r and outgoing direction a:
     F[r*n_ang + a] = k^2 e^{i d gamma} h^d sum_j e^{-i k z_j.alpha_a}
                      chi_j (u_in,r,j + u_r,j).
   u_dev: c128 n_rhs x m^d (from csff_solve); alpha_host: n_ang x dim.
   F_dev: c128 n_rhs x n_ang (device).  F_exp_dev: int32 n_rhs x n_ang
   (device) or NULL.  With F_exp_dev the true value is F * 2^F_exp, which
   keeps maps whose terms exceed the FP64 range finite; without it F is the
   plain value (Inf where it does not fit) and the call returns
   CSFF_WARN_ILL_CONDITIONED if any scale was needed.  Arithmetic: FP64. */
csff_status csff_far_field(csff_plan* plan, int n_rhs, const double* eta_host, const void* u_dev,
                           int n_ang, const double* alpha_host, void* F_dev, int32_t* F_exp_dev);

/* Arithmetic of the far-field contraction (eq. FFmap; the paper leaves the
   quadrature's arithmetic open, Sec. 4).
   CSFF_FF_FP64 (default): FP64-class throughout (2D stage 1 in double-float
     arithmetic on the FP32 pipes, FP64 where the operand ranges need it).
   CSFF_FF_TC_BF16X4: 3D plans evaluate the z-contraction (the largest stage)
     on the tensor cores: each operand split into four BF16 terms (32
     significant bits), the ten products of terms i, j with i + j <= 3
     accumulated in FP32 over 32 z-nodes at a time and summed in double-float
     across them; F then carries an absolute error of about 2^-26 times
     sum_j |term_j| per angle.  The library falls back to FP64 on the device
     when an operand is not finite or its exponent range is too wide.  2D plans
     are unaffected.  A wait inside the tensor-core kernel that runs out makes
     csff_far_field return CSFF_ERR_TIMEOUT.
   Errors: CSFF_ERR_INVALID_ARG for an unknown mode. */
enum { CSFF_FF_FP64 = 0, CSFF_FF_TC_BF16X4 = 1 };
csff_status csff_plan_set_far_field_mode(csff_plan* plan, int mode);

/* The 2D far field's stage-1 contraction skips the 32-node blocks whose
   terms, bounded through per-block exponents, stay below 2^-55 of the sum of
   the magnitudes of each far-field value's terms (Sec. 3.3: on the rotated
   contour the terms span hundreds of orders of magnitude, so most blocks of a
   large-k map are negligible).  *executed (host) receives the fraction of the
   contraction's work the plan's last 2D far field carried out (1 for 3D
   plans, for the FP64 range-fallback kernel, or before any far field).
   Synchronises the plan's stream.  Errors: CSFF_ERR_INVALID_ARG, CSFF_ERR_CUDA. */
csff_status csff_far_field_work(csff_plan* plan, double* executed);

/* ---- user coefficients and right-hand sides (Sec. 5.2-5.3) ---------------
   The partial-wave Schroedinger problem (-1/2 Delta + V - E) u = phi along the
   rotated contour is, times 2, the plan's operator A u = c (2d u - sum_nbr u)
   - q u with q = 2E - 2V and right-hand side 2 phi; its potentials are not
   Gaussians of the kind csff_problem describes, so they are given as samples. */

/* Replace the plan's q = k^2 (1 + chi) by samples of q at the finest level's
   interior nodes (q_dev: device, complex128, m^d values, x fastest; read
   during the call).  Coarser levels take q at their nodes (injection: coarse
   nodes are fine nodes), 1/d and the FP32 copies are rebuilt and the coarsest
   inverse is formed again (FP64 Gauss-Jordan on the host).  From then on
   V-cycles use the per-level kernels (the fused FP32 tiles form q from the
   Gaussian factors).  csff_rhs / csff_solve keep forming the Gaussian
   right-hand side; use csff_solve_rhs.  Errors: CSFF_ERR_INVALID_ARG for NULL
   arguments or a singular coarsest operator, CSFF_ERR_CUDA. */
csff_status csff_plan_set_potential(csff_plan* plan, const void* q_dev);

/* Solve A u = b for one right-hand side b_dev (device, complex128, m^d
   values, read only) into u_dev (device, complex128, m^d; the initial guess
   when use_guess != 0, else ignored), with the plan's smoother, precision and
   tolerance; info (host, may be NULL) as for csff_solve.  Returns the solve's
   status (CSFF_ERR_NOT_CONVERGED, CSFF_ERR_DIVERGED, CSFF_ERR_NONFINITE are
   reported with u holding the last iterate). */
csff_status csff_solve_rhs(csff_plan* plan, const void* b_dev, void* u_dev, int use_guess, csff_info* info);

/* The partial-wave Schroedinger problem of Sec. 5.2, eq. (partialwave2d),
   (-1/2 Delta + V - E) u = phi on the rotated contour, multiplied by 2: the
   plan's operator with q = 2E - 2V and the right-hand side 2 phi.
   csff_plan_set_schroedinger forms q on the device from the samples V_dev
   (device, complex128, m^d values at the finest level's interior nodes, x
   fastest: V = V1 + V2 + V12 at z; read during the call) and then proceeds as
   csff_plan_set_potential.  csff_solve_schroedinger forms b = 2 phi from
   phi_dev (device, complex128, m^d, read only) and proceeds as
   csff_solve_rhs.  Errors: CSFF_ERR_INVALID_ARG (NULL arguments, E not
   finite, singular coarsest operator), CSFF_ERR_CUDA; solve statuses as for
   csff_solve_rhs. */
csff_status csff_plan_set_schroedinger(csff_plan* plan, double E, const void* V_dev);
csff_status csff_solve_schroedinger(csff_plan* plan, const void* phi_dev, void* u_dev, int use_guess,
                                    csff_info* info);

/* One-dimensional functions along the contour z_i = i h e^{i gamma},
   i = 1 .. m (zero at i = 0 and i = m + 1), with the three-point stencil of
   -1/2 d^2/dz^2; v (host, 2m doubles, interleaved re/im) holds V(z_i).

   Bound state of eq. (boundstate), (-1/2 d^2/dz^2 + V) phi = lambda phi: the
   eigenpair nearest lambda_guess, by inverse iteration with the fixed shift
   followed by Rayleigh-quotient updates (bilinear form, no conjugate: the
   contour operator is complex symmetric).  phi (host, 2m doubles) is scaled
   so that sum_i phi_i^2 h e^{i gamma} = 1 and its largest entry has a
   non-negative real part; lambda (host, 2 doubles).  Errors:
   CSFF_ERR_INVALID_ARG, CSFF_ERR_NOT_CONVERGED after 200 steps. */
csff_status csff_contour_bound_state(int m, double h, double gamma, const double* v, double lambda_guess,
                                     double* lambda, double* phi);

/* Regular solution of eq. (testfunction), (-1/2 d^2/dz^2 + V - k^2/2) phi = 0
   with phi = 0 at z = 0, by the recurrence of the discrete equation, scaled
   to sin(kappa z + delta) / sqrt(k) where |V| < tail (kappa: the discrete
   wavenumber, cos(kappa h e^{i gamma}) = 1 - (k h e^{i gamma})^2 / 2; the
   scale is fitted at the first two such nodes).  phi: host, 2m doubles.
   Errors: CSFF_ERR_INVALID_ARG (also when |V| never falls below tail). */
csff_status csff_contour_regular_solution(int m, double h, double gamma, const double* v, double k, double tail,
                                          double* phi);

/* Separable contour integrals of eqs. (single-ionization) and
   (double-ionization) on a 2D plan:
     out[r] = e^{2 i gamma} h^2 sum_{j,i} X[r][i] Y[r][j] (f - w u)[j][i],
   r < n_rows, i the x index and j the y index of the finest level's interior
   nodes.  X, Y: device, complex128, n_rows x m, row-major; f, w, u: device,
   complex128, m x m (x fastest); w and u both NULL means the integrand f;
   out: device, complex128, n_rows.  Runs on the plan's stream (FP64).
   Errors: CSFF_ERR_INVALID_ARG (3D plan, NULL buffers, only one of w, u),
   CSFF_ERR_CUDA. */
csff_status csff_separable_sum(csff_plan* plan, int n_rows, const void* X, const void* Y, const void* f,
                               const void* w, const void* u, void* out);

/* ---- per-step calls (one kernel each; for verification and custom cycles) --
   arith: CSFF_ARITH_FP64 (c128 buffers) or CSFF_ARITH_FP32 (c64 buffers).
   level: 0 = finest.  All buffers are device pointers of m_level^d elements
   unless stated.  Coefficients are the plan's (FP32 copies for FP32). */

/* K1: r = b - A_l u (eq. csg with the Sec. 5.2 stencil). */
csff_status csff_residual(csff_plan* plan, int level, int arith, const void* u_dev,
                          const void* b_dev, void* r_dev);
/* K2: `sweeps` sweeps of the plan's smoother on A_l u = b, in place on u_dev.
   Jacobi: u <- u + omega D^{-1}(b - A u) (uses a plan buffer for the new
   iterate).  RBGS: red points (even sum of node indices) then black. */
csff_status csff_smooth(csff_plan* plan, int level, int arith, void* u_dev, const void* b_dev,
                        int sweeps);
/* K3: b_c (level+1) = full weighting of r_f (level). */
csff_status csff_restrict(csff_plan* plan, int level, int arith, const void* r_fine_dev,
                          void* b_coarse_dev);
/* K4: u_f (level) += bi/trilinear interpolation of e_c (level+1). */
csff_status csff_prolong_add(csff_plan* plan, int level, int arith, const void* e_coarse_dev,
                             void* u_fine_dev);
/* K5: u_c = A_c^{-1} b_c on the coarsest level.  The inverse is formed in
   FP64; FP64: FP64 product; FP32: the inverse rounded to FP32, FP32 product.
   Buffers in the precision given by arith. */
csff_status csff_coarse_solve(csff_plan* plan, int arith, const void* b_dev, void* u_dev);
/* K6: ||v||_2 over m_level^d complex values, accumulated in FP64; result in
   *out_host (synchronises the stream). */
csff_status csff_norm2(csff_plan* plan, int level, int arith, const void* v_dev, double* out_host);
/* One V(nu1, nu2) cycle on the finest level, in place on u_dev. */
csff_status csff_vcycle(csff_plan* plan, int arith, void* u_dev, const void* b_dev);

/* ---- learned smoother --------------------------------------------------
   Not in the paper: a bias-free 3x3 convolutional network N (2 -> 16 -> 16 ->
   2 channels, ReLU between layers) on the two real channels of a residual,
   used as u <- u + N(h^2 (b - A u)) after each red-black sweep of the FP32
   cycles on the finest levels.  Weights and activations BF16, FP32 accumulation, FP32
   master weights.  Weight layout: flat (out, in, a, b) per layer, layers 1, 2,
   3 (288 + 2304 + 288 = 2880 values).  Convolutions are 3x3
   cross-correlations with zero padding.  Training (all on the GPU): loss
   L = mean over patches of sum_mask |r - A N(r)|^2 / sum_mask |r|^2, A the
   level's operator with per-pixel q = k^2(1 + chi) and constant c (eq. csg),
   mask = interior minus a margin; Adam (beta 0.9/0.999, eps 1e-8). */
typedef struct csff_net csff_net;
int csff_net_num_params(void);
/* w_host: 2880 FP32 weights (copied). */
csff_status csff_net_create(const float* w_host, csff_net** out);
void csff_net_destroy(csff_net* net);
csff_status csff_net_set_weights(csff_net* net, const float* w_host);   /* resets Adam state */
csff_status csff_net_get_weights(const csff_net* net, float* w_host);
/* y_dev = N(r_dev) for B patches of H x W (c64 each, device). */
csff_status csff_net_forward(csff_net* net, int B, int H, int W, const void* r_dev, void* y_dev, void* stream);
/* The same forward pass over the warp-level MMA tile (mma.sync, no tensor
   memory), the form the batched persistent kernel runs; results agree with
   csff_net_forward to the accumulation order. */
csff_status csff_net_forward_mma(csff_net* net, int B, int H, int W, const void* r_dev, void* y_dev, void* stream);
/* Loss and FP32 weight gradient of a batch: r_dev, q_dev c64 [B][H][W];
   c_host: B complex constants (re, im); grad_host: 2880 floats or NULL. */
csff_status csff_net_loss_grad(csff_net* net, int B, int H, int W, const void* r_dev, const void* q_dev,
                               const double* c_host, int margin, float* loss_host, float* grad_host, void* stream);
/* One Adam step on a batch (loss before the step in *loss_host if non-NULL). */
csff_status csff_net_train_step(csff_net* net, int B, int H, int W, const void* r_dev, const void* q_dev,
                                const double* c_host, int margin, float lr, float* loss_host, void* stream);
/* The 3D network: the same three layers with 3x3x3 cross-correlations
   (out[o][z][y][x] = sum_c sum_{a,b,e} w[o][c][a][b][e] x[c][z+a-1][y+b-1][x+e-1],
   zero padding), weights flat (out, in, a, b, e): 864 + 6912 + 864 = 8640
   values; its loss takes the 7-point operator A y = c (6 y - sum_nbr y) - q y.
   Patches [B][Z][H][W], c64.  Same precision and training as the 2D network;
   csff_net_set_weights, _get_weights and _destroy serve both.  A network of
   one dimension is refused (CSFF_ERR_INVALID_ARG) by the other dimension's
   calls and by plans of the other dimension. */
int csff_net_num_params3(void);
csff_status csff_net_create3(const float* w_host, csff_net** out);
csff_status csff_net_forward3(csff_net* net, int B, int Z, int H, int W, const void* r_dev, void* y_dev, void* stream);
csff_status csff_net_loss_grad3(csff_net* net, int B, int Z, int H, int W, const void* r_dev, const void* q_dev,
                                const double* c_host, int margin, float* loss_host, float* grad_host, void* stream);
csff_status csff_net_train_step3(csff_net* net, int B, int Z, int H, int W, const void* r_dev, const void* q_dev,
                                 const double* c_host, int margin, float lr, float* loss_host, void* stream);
/* Attach (net != NULL) or detach the learned step on levels 0..levels-1 of a
   red-black plan's FP32 cycles (mixed-precision solves): after each red-black
   sweep, u <- u + N(h_l^2 r) with r the level's residual (so the network sees
   the operator in units of h^2, O(1) on every grid); 2D plans take a 2D
   network, 3D plans a 3D one.  The first two
   refinement steps of each solve run plain red-black sweeps; the second sets
   the reference reduction factor f = min(its factor, guard); a later learned step
   that reduces the residual by less than f turns the learned step off for the
   rest of that solve (csff_info.flags bit 1); with adaptive_inner the
   factors are taken per inner_cycles cycles, f^(inner_cycles / cycles of the
   step).  The plan keeps a pointer to the net; the net must outlive the
   attachment. */
csff_status csff_plan_set_learned(csff_plan* plan, csff_net* net, int levels, double guard);
/* Use net (NULL: the plan's network again) for the learned step on one level
   0 <= level < levels of the last csff_plan_set_learned.  In units of h^2 a
   level's operator depends on k h, which doubles from one level to the next,
   so a coarser level is served by a network trained at its own k h.
   csff_plan_set_learned clears these replacements.  Errors:
   CSFF_ERR_INVALID_ARG (no learned step on that level), CSFF_ERR_OOM. */
csff_status csff_plan_set_learned_level(csff_plan* plan, int level, csff_net* net);
/* FP32 copy of a level's q = k^2(1 + chi) (c64, m_l^d, device) and its
   constant c = e^{-2i gamma}/h_l^2 (2 doubles, host): the operator the learned
   step is trained against. */
csff_status csff_plan_copy_coefficients(const csff_plan* plan, int level, void* q32_dev, double* c_host);

/* ---- batched solve: many uneven 2D problems in one persistent launch ----
   Each instance runs the refinement loop of CSFF_PREC_MIXED with the FP64
   residual and update of its own kernel (FP32 V(1,1) red-black cycles on the
   scaled correction with the coarsest solve in FP64; Sec. 4 with the
   refinement loop; inner_cycles per step, or with adaptive_inner each
   instance's steps sized from its previous step's reduction factor as in the
   single-plan solve; refine_fp64 is ignored), but all instances advance inside
   one cooperative kernel whose phases are separated by grid barriers; the
   tiles of every active instance are shared out among the CTAs, convergence
   is decided per instance on the device.  The solve is captured once as a
   CUDA graph and replayed.  Barrier waits are bounded: a wait that runs out
   ends the kernel with CSFF_ERR_TIMEOUT (no trap, no hang).
   Requirements: dim = 2, red-black GS, nu1 = nu2 = 1, precision MIXED,
   n >= 65, at most 12 levels; otherwise CSFF_ERR_UNSUPPORTED. */
typedef struct csff_batch csff_batch;
/* probs: n_inst problems (host, copied); opts: shared by all instances. */
csff_status csff_batch_create(int n_inst, const csff_problem* probs, const csff_opts* opts, void* stream,
                              csff_batch** out);
void csff_batch_destroy(csff_batch* batch);
/* eta_host: n_inst x 2 incident directions; infos_host: n_inst reports or NULL.
   Synchronises.  Returns the worst instance status. */
csff_status csff_batch_solve(csff_batch* batch, const double* eta_host, csff_info* infos_host);
/* Device pointer (c128, m_i^2) to instance i's solution of the last solve;
   owned by the batch, valid until the next solve. */
csff_status csff_batch_solution(const csff_batch* batch, int i, const void** u_dev);
/* Copy of instance i's solution into the caller's u_out_dev (c128, m_i^2);
   synchronises the batch's stream. */
csff_status csff_batch_copy_solution(const csff_batch* batch, int i, void* u_out_dev);
/* Far-field map of every instance (as csff_far_field): n_ang[i] directions
   alpha_host[i] (host, n_ang[i] x 2) into F_dev[i] (c128) and, if F_exp_dev
   is not NULL, the exponents F_exp_dev[i] (int32). */
csff_status csff_batch_far_field(csff_batch* batch, const double* eta_host, const int* n_ang,
                                 const double* const* alpha_host, void* const* F_dev, int32_t* const* F_exp_dev);
/* Autotuner: times the persistent solve for each tile size of the large
   levels (16 or 8 coarse points per tile side) and each CTA count per SM the
   occupancy allows, keeps the fastest; chosen values returned if non-NULL. */
csff_status csff_batch_autotune(csff_batch* batch, const double* eta_host, int* tc_big_out, int* ctas_per_sm_out);
/* Fix the tile choice by hand instead: tc_big = 16 or 8 coarse points per
   tile side on the levels with at least 64 coarse points per side (16 is the
   choice before any autotune), ctas_per_sm = CTAs per SM of the persistent
   launch (0 = the occupancy maximum, larger values are clamped to it).
   Errors: CSFF_ERR_INVALID_ARG. */
csff_status csff_batch_set_tiles(csff_batch* batch, int tc_big, int ctas_per_sm);
/* Learned smoother in the batched solve (an addition to the paper's method,
   like csff_plan_set_learned): every FP32 V-cycle of an instance ends with
   u <- u + N(h^2 (b - A u)) on its finest level, N the network (not owned; it
   must outlive the solves that use it, and its weights are read at each
   solve).  The first two refinement steps of an instance run without it; the
   second's reduction factor, capped at guard, is the reference; an instance
   whose learned step reduces the residual less than the reference runs plain
   cycles for the rest of its solve (info.flags bit 1; bit 0 = a network was
   set); with adaptive_inner the factors are taken per inner_cycles cycles, as
   in the single-problem solve.  net = NULL removes it.  Errors: CSFF_ERR_INVALID_ARG (guard <= 0, or the network's
   shared memory does not fit beside the tiles'). */
csff_status csff_batch_set_learned(csff_batch* batch, csff_net* net, double guard);

/* Test hook for the bounded barrier: extra_arrivals = 1 makes every grid
   barrier of the next solves wait for one CTA that does not exist, so each
   wait runs out after spin_limit polls (0 = the default limit of 2^26 polls
   of ~64 ns) and the solve returns CSFF_ERR_TIMEOUT; 0 restores normal runs. */
csff_status csff_batch_debug_barrier(csff_batch* batch, int extra_arrivals, long long spin_limit);

/* Allocation-free Euclidean norm.  The paper has no counterpart: this is a
   service for callers that cannot allocate device memory (memory owned by
   another allocator, or loops that must not pay cudaMalloc's implicit device
   synchronisation).  Needs no plan and calls no cudaMalloc/cudaFree.
     *out_dev (device double) = 2^exp_scale * sqrt(sum |v_j 2^-exp_scale|^2)
   over n complex values v_dev (c128 for CSFF_ARITH_FP64, c64 for FP32),
   accumulated in FP64; enqueued on `stream` (a cudaStream_t, NULL = legacy
   default), nothing is synchronised.  exp_scale in [-1000, 1000] guards the
   squares against overflow (pass 0 for ordinary magnitudes).
   Scratch: a fixed 32 KiB device array inside the library (4096 per-block
   partial sums), held by every GPU that loads the library until exit;
   n is limited to 33554432 (2^25) values, larger n returns
   CSFF_ERR_INVALID_ARG with a message.  All calls share that array: calls
   whose work overlaps on the GPU (different streams, or different host
   threads on one device) race and give wrong results; serialise them.
   The first call on each device looks up the array's device address
   (cudaGetSymbolAddress, with that device current) and keeps it with the id
   of the device's current CUDA context; a call that finds another context
   there (after cudaDeviceReset, say) looks the address up again.  Make the
   first call on a device, and the first after such a reset, before any
   stream capture.  v_dev and out_dev must be addresses in the calling
   thread's current context. */
csff_status csff_norm2_noalloc(int arith, const void* v_dev, long long n, int exp_scale, double* out_dev,
                               void* stream);

/* ---- measurement --------------------------------------------------------
   While recording, the library brackets every launch of the selected kernel
   families with a pair of CUDA events on the launching stream and adds up
   the algorithmic bytes (arrays each kernel must read and write; per-point
   coefficient tables excluded, since they can be rebuilt from O(n) tables)
   and flops of those launches.  Global to the process, not thread-safe. */
enum {
  CSFF_PROF_FF_CONTRACT = 1, /* far-field stage-1 contraction (FP64) */
  CSFF_PROF_MG32 = 2,        /* multigrid kernels in FP32 */
  CSFF_PROF_MG64 = 4,        /* multigrid kernels in FP64 and the mixed solve's
                                double-float refinement kernels */
  CSFF_PROF_FF_OTHER = 8,    /* far-field tables, g field, stage 2 */
  CSFF_PROF_TILES32 = 16,    /* the fused FP32 V(1,1) tile kernels alone (also counted in MG32) */
  CSFF_PROF_TILES32_FINE = 32 /* those of them that work on a plan's finest level (also in TILES32) */
};
#define CSFF_PROF_FAMILIES 6
typedef struct csff_prof_stats {
  int launches;
  double ms;          /* summed event time of the launches */
  double alg_bytes;   /* summed algorithmic bytes */
  double alg_flops;   /* summed algorithmic real flops */
} csff_prof_stats;
csff_status csff_prof_begin(unsigned family_mask);
/* Stop recording, wait for the recorded events, write one entry per family
   (index log2 of the family bit) to out_host[CSFF_PROF_FAMILIES]. */
csff_status csff_prof_end(csff_prof_stats* out_host);

/* ---- helpers ------------------------------------------------------------ */

/* eq. (thetagamma): gamma = atan(sin theta / (2 + cos theta)). */
double csff_gamma_from_ecs(double theta_ecs);
/* The adaptive refinement schedule (csff_opts.adaptive_inner): after a step of
   cycles_run FP32 V-cycles took the relative residual from rel_before to
   rel_after, the next step runs n = ceil(log(rel_tol / rel_after) / log rho
   - 1e-9) cycles, rho = (rel_after / rel_before)^(1 / cycles_run) the per-cycle
   reduction factor, clamped to [1, max_cycles].  Without a reduction
   (rel_after >= rel_before, or a non-positive or non-finite value) it returns
   max_cycles; max_cycles < 1 counts as 1.  Host only. */
int csff_refinement_cycles(double rel_before, double rel_after, int cycles_run, double rel_tol, int max_cycles);
const char* csff_status_string(csff_status s);
const char* csff_last_error(void);
/* Number of CUDA kernel launches the library made in this process. */
uint64_t csff_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* CSFF_H */
