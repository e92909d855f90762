// C ABI of libcsff: plan construction, the multigrid solve drivers (FP64 and
// FP32-inner / double-float refinement), the far-field call and the per-step
// calls.
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "csff_internal.h"

using csff::cx;
using csff::Level;

namespace csff {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_last_error;

void set_error(const std::string& s) { t_last_error = s; }

csff_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? CSFF_ERR_OOM : CSFF_ERR_CUDA;
}

// ---- kernel-family timing (csff_prof_begin / csff_prof_end) -------------------
namespace {
struct ProfRec {
  int family;
  cudaEvent_t a, b;
  double bytes, flops;
};
struct ProfState {
  unsigned mask = 0;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
ProfState g_prof;
}  // namespace

thread_local bool g_capturing = false;   // this thread is capturing a graph (plans may run on several threads)
unsigned prof_mask() { return g_prof.mask; }

// the record list is shared by every thread that launches while profiling is on
std::mutex g_prof_mu;

ProfScope::ProfScope(int family, cudaStream_t s, double bytes, double flops, int family2, int family3)
    : stream(s) {
  if (g_capturing) return;
  const bool on1 = (g_prof.mask & (1u << family)) != 0;
  const bool on2 = family2 >= 0 && (g_prof.mask & (1u << family2)) != 0;
  const bool on3 = family3 >= 0 && (g_prof.mask & (1u << family3)) != 0;
  if (!on1 && !on2 && !on3) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  auto add = [&](int f) {
    ProfRec r{f, g_prof.get(), g_prof.get(), bytes, flops};
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, s);
    g_prof.recs.push_back(r);
    return (int)g_prof.recs.size() - 1;
  };
  if (on1) slot = add(family);
  if (on2) slot2 = add(family2);
  if (on3) slot3 = add(family3);
}

ProfScope::~ProfScope() {
  if (slot < 0 && slot2 < 0 && slot3 < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot >= 0) cudaEventRecord(g_prof.recs[slot].b, stream);
  if (slot2 >= 0) cudaEventRecord(g_prof.recs[slot2].b, stream);
  if (slot3 >= 0) cudaEventRecord(g_prof.recs[slot3].b, stream);
}

}  // namespace csff

namespace {

using cd = std::complex<double>;

#define CK(call, what)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return csff::cuda_fail(e_, what);        \
  } while (0)

#define CS(call)                                                    \
  do {                                                              \
    csff_status s_ = (call);                                        \
    if (s_ != CSFF_OK) return s_;                                   \
  } while (0)

csff_status invalid(const std::string& s) {
  csff::set_error(s);
  return CSFF_ERR_INVALID_ARG;
}

template <typename P>
csff_status dev_alloc(csff_plan* plan, P** p, size_t count) {
  size_t bytes = sizeof(P) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return csff::cuda_fail(e, "cudaMalloc");
  }
  plan->bytes += bytes;
  return CSFF_OK;
}

// chi per axis at the interior nodes of a grid with n nodes:
// E_{g,c}(i) = exp(-(x_i e^{i gamma} - center_c)^2 / w), amplitude folded into c = 0.
std::vector<double2> chi_tables(const csff_plan* P, int n) {
  const int d = P->dim, m = n - 2, G = P->prob.n_gauss;
  const double h = (P->prob.box_hi - P->prob.box_lo) / (n - 1);
  const cd rot = std::polar(1.0, P->prob.gamma);
  std::vector<double2> t((size_t)G * d * m);
  for (int g = 0; g < G; ++g) {
    const csff_gauss& q = P->gauss[g];
    for (int c = 0; c < d; ++c)
      for (int i = 0; i < m; ++i) {
        double x = P->prob.box_lo + (i + 1) * h;
        cd z = x * rot - q.center[c];
        cd v = std::exp(-z * z / q.width);
        if (c == 0) v *= cd(q.amp_re, q.amp_im);
        t[((size_t)g * d + c) * m + i] = make_double2(v.real(), v.imag());
      }
  }
  return t;
}

// FP32 factors of q for the fused 2D tiles: per Gaussian X = k^2 t_x (t_x
// carries the amplitude), Y = t_y, rescaled by 2^-s and 2^s so that the two
// factors' largest magnitudes agree (the product is unchanged; neither factor
// leaves FP32's range unless q itself does).
std::vector<float2> fp32_factors(const csff_plan* P, const std::vector<double2>& tab, int m) {
  const int G = P->prob.n_gauss;
  const double k2 = P->prob.k * P->prob.k;
  std::vector<float2> out((size_t)G * 2 * m);
  for (int g = 0; g < G; ++g) {
    const double2* tx = &tab[((size_t)g * 2) * m];
    const double2* ty = &tab[((size_t)g * 2 + 1) * m];
    double mx = 0, my = 0;
    for (int i = 0; i < m; ++i) {
      mx = std::max(mx, k2 * std::hypot(tx[i].x, tx[i].y));
      my = std::max(my, std::hypot(ty[i].x, ty[i].y));
    }
    int sh = 0;
    if (mx > 0 && my > 0) sh = (int)std::lround(0.5 * (std::log2(mx) - std::log2(my)));
    for (int i = 0; i < m; ++i) {
      out[((size_t)g * 2) * m + i] =
          make_float2((float)std::ldexp(k2 * tx[i].x, -sh), (float)std::ldexp(k2 * tx[i].y, -sh));
      out[((size_t)g * 2 + 1) * m + i] = make_float2((float)std::ldexp(ty[i].x, sh), (float)std::ldexp(ty[i].y, sh));
    }
  }
  return out;
}

// Dense inverse of the coarsest operator by LU with partial pivoting.
// qv: the coarsest level's q from user samples (else formed from the Gaussians)
bool coarse_inverse(const csff_plan* P, const Level& L, std::vector<double2>& out,
                    const std::vector<double2>* qv = nullptr) {
  const int d = P->dim, m = L.m;
  const int N = (d == 3) ? m * m * m : m * m;
  std::vector<double2> tab = chi_tables(P, L.n);
  const int G = P->prob.n_gauss;
  const double k2 = P->prob.k * P->prob.k;
  const cd c(L.c.x, L.c.y);
  std::vector<cd> A((size_t)N * N, cd(0, 0));
  auto id = [&](int ix, int iy, int iz) { return (iz * m + iy) * m + ix; };
  for (int iz = 0; iz < (d == 3 ? m : 1); ++iz)
    for (int iy = 0; iy < m; ++iy)
      for (int ix = 0; ix < m; ++ix) {
        cd chi(0, 0);
        for (int g = 0; g < G; ++g) {
          const double2* t = &tab[(size_t)g * d * m];
          cd v = cd(t[ix].x, t[ix].y) * cd(t[m + iy].x, t[m + iy].y);
          if (d == 3) v *= cd(t[2 * m + iz].x, t[2 * m + iz].y);
          chi += v;
        }
        int r = id(ix, iy, iz);
        A[(size_t)r * N + r] = qv ? 2.0 * d * c - cd((*qv)[r].x, (*qv)[r].y) : 2.0 * d * c - k2 * (1.0 + chi);
        int nb[6][3] = {{ix - 1, iy, iz}, {ix + 1, iy, iz}, {ix, iy - 1, iz},
                        {ix, iy + 1, iz}, {ix, iy, iz - 1}, {ix, iy, iz + 1}};
        for (int q = 0; q < 2 * d; ++q) {
          int a = nb[q][0], b = nb[q][1], e = nb[q][2];
          if (a < 0 || a >= m || b < 0 || b >= m || e < 0 || e >= (d == 3 ? m : 1)) continue;
          A[(size_t)r * N + id(a, b, e)] = -c;
        }
      }
  // Gauss-Jordan on [A | I] with partial pivoting
  std::vector<cd> I((size_t)N * N, cd(0, 0));
  for (int i = 0; i < N; ++i) I[(size_t)i * N + i] = 1.0;
  for (int col = 0; col < N; ++col) {
    int piv = col;
    for (int r = col + 1; r < N; ++r)
      if (std::abs(A[(size_t)r * N + col]) > std::abs(A[(size_t)piv * N + col])) piv = r;
    if (std::abs(A[(size_t)piv * N + col]) == 0.0) return false;
    if (piv != col)
      for (int j = 0; j < N; ++j) {
        std::swap(A[(size_t)piv * N + j], A[(size_t)col * N + j]);
        std::swap(I[(size_t)piv * N + j], I[(size_t)col * N + j]);
      }
    cd inv = 1.0 / A[(size_t)col * N + col];
    for (int j = 0; j < N; ++j) {
      A[(size_t)col * N + j] *= inv;
      I[(size_t)col * N + j] *= inv;
    }
    for (int r = 0; r < N; ++r) {
      if (r == col) continue;
      cd f = A[(size_t)r * N + col];
      if (f == cd(0, 0)) continue;
      for (int j = 0; j < N; ++j) {
        A[(size_t)r * N + j] -= f * A[(size_t)col * N + j];
        I[(size_t)r * N + j] -= f * I[(size_t)col * N + j];
      }
    }
  }
  out.resize((size_t)N * N);
  for (size_t i = 0; i < out.size(); ++i) out[i] = make_double2(I[i].real(), I[i].imag());
  return true;
}

// Incident-wave tables U_c(i) = exp(i k eta_c x_i e^{i gamma}) on the finest grid.
csff_status upload_uinc(csff_plan* P, const double* eta) {
  const Level& L = P->lv[0];
  const int d = P->dim, m = L.m;
  std::vector<double2> ut((size_t)d * m);
  const cd ik(0.0, P->prob.k), rot = std::polar(1.0, P->prob.gamma);
  for (int c = 0; c < d; ++c)
    for (int i = 0; i < m; ++i) {
      double x = P->prob.box_lo + (i + 1) * L.h;
      cd v = std::exp(ik * eta[c] * x * rot);
      ut[(size_t)c * m + i] = make_double2(v.real(), v.imag());
    }
  CK(cudaMemcpyAsync(P->uinc_tab, ut.data(), sizeof(double2) * ut.size(), cudaMemcpyHostToDevice, P->stream),
     "upload incident tables");
  return CSFF_OK;
}

// ---- per-precision buffer access ------------------------------------------------
template <typename T> cx<T>* ubuf(Level& L);
template <> double2* ubuf<double>(Level& L) { return L.u64; }
template <> float2* ubuf<float>(Level& L) { return L.u32; }
template <typename T> cx<T>* tbuf(Level& L);
template <> double2* tbuf<double>(Level& L) { return L.t64; }
template <> float2* tbuf<float>(Level& L) { return L.t32; }
template <typename T> const cx<T>* cinv(const csff_plan* P);
template <> const double2* cinv<double>(const csff_plan* P) { return P->coarse_inv; }
template <> const float2* cinv<float>(const csff_plan* P) { return P->coarse_inv32; }
template <typename T> cx<T>* bbuf(Level& L);
template <> double2* bbuf<double>(Level& L) { return L.b64; }
template <> float2* bbuf<float>(Level& L) { return L.b32; }
template <typename T> cx<T>* rbuf(Level& L);
template <> double2* rbuf<double>(Level& L) { return L.r64; }
template <> float2* rbuf<float>(Level& L) { return L.r32; }

// The mixed solve with the FP64 refinement applies the coarsest inverse in
// FP64 inside its FP32 cycles: FP64 for the outer residual, the update and the
// coarsest-grid solve, FP32 for the rest of the cycle.
bool coarse_fp64(const csff_plan* P) { return P->opts.precision == CSFF_PREC_MIXED && P->opts.refine_fp64 != 0; }

template <typename T>
csff_status smooth(csff_plan* P, int l, cx<T>* u, const cx<T>* b, int sweeps) {
  Level& L = P->lv[l];
  cudaStream_t s = P->stream;
  if (P->opts.smoother == CSFF_SMOOTHER_GMRES) {
    for (int i = 0; i < sweeps; ++i)
      CK(csff::launch_gmres_step<T>(P->dim, L, P->opts.krylov_m, u, b, reinterpret_cast<cx<T>*>(P->gm_v),
                                    P->gm_part, P->red_blocks, P->gm, s),
         "gmres");
    return CSFF_OK;
  }
  if (P->opts.smoother == CSFF_SMOOTHER_RBGS) {
    for (int i = 0; i < sweeps; ++i) {
      CK(csff::launch_rbgs<T>(P->dim, L, u, b, s), "rbgs");
      if constexpr (sizeof(T) == 4) {
        if (P->net && !P->learned_off && l < P->learned_levels) CS(csff::learned_step(P, l, P->dim, L, u, b, s));
      }
    }
    return CSFF_OK;
  }
  cx<T>* t = tbuf<T>(L);
  int i = 0;
  for (; i + 1 < sweeps; i += 2) {
    CK(csff::launch_jacobi<T>(P->dim, L, P->opts.omega, u, b, t, s), "jacobi");
    CK(csff::launch_jacobi<T>(P->dim, L, P->opts.omega, t, b, u, s), "jacobi");
  }
  if (i < sweeps) {
    CK(csff::launch_jacobi<T>(P->dim, L, P->opts.omega, u, b, t, s), "jacobi");
    CK(cudaMemcpyAsync(u, t, sizeof(cx<T>) * (size_t)L.N, cudaMemcpyDeviceToDevice, s), "copy");
  }
  return CSFF_OK;
}

// One V(nu1, nu2) cycle on level l for A_l u = b (Sec. 4).
template <typename T>
csff_status vcycle(csff_plan* P, int l, cx<T>* u, const cx<T>* b) {
  const int nl = (int)P->lv.size();
  cudaStream_t s = P->stream;
  if (l == nl - 1) {
    if constexpr (sizeof(T) == 4) {
      if (coarse_fp64(P)) {
        CK(csff::launch_coarse_solve_f64(P->coarse_inv, P->coarse_N, b, u, s), "coarse solve");
        return CSFF_OK;
      }
    }
    CK(csff::launch_coarse_solve<T>(cinv<T>(P), P->coarse_N, b, u, s), "coarse solve");
    return CSFF_OK;
  }
  Level& L = P->lv[l];
  Level& C = P->lv[l + 1];
  CS(smooth<T>(P, l, u, b, P->opts.nu1));
  CK(csff::launch_residual<T>(P->dim, L, u, b, rbuf<T>(L), s), "residual");
  CK(csff::launch_restrict<T>(P->dim, L, C, rbuf<T>(L), bbuf<T>(C), s), "restrict");
  if (l + 1 < nl - 1) CK(csff::launch_zero<T>(ubuf<T>(C), C.N, s), "zero");
  CS(vcycle<T>(P, l + 1, ubuf<T>(C), bbuf<T>(C)));
  CK(csff::launch_prolong_add<T>(P->dim, L, C, ubuf<T>(C), u, s), "prolong");
  CS(smooth<T>(P, l, u, b, P->opts.nu2));
  return CSFF_OK;
}

// norm of a level-0 FP64 vector into red_out[slot] (device), scaled by 2^-e.
csff_status norm64(csff_plan* P, const double2* v, int e, int slot) {
  CK(csff::launch_norm2<double>(v, P->lv[0].N, e, P->red, P->red_blocks, P->red_out + slot, P->stream),
     "norm");
  return CSFF_OK;
}

csff_status read_scalars(csff_plan* P, int count) {
  CK(cudaMemcpyAsync(P->red_host, P->red_out, sizeof(double) * count, cudaMemcpyDeviceToHost, P->stream),
     "read norms");
  CK(cudaStreamSynchronize(P->stream), "sync");
  return CSFF_OK;
}

struct Tracker {
  csff_info* info;
  double prev = 0;
  int rises = 0;
  void start(csff_info* in) {
    info = in;
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->history[0] = 1.0;
      info->n_hist = 1;
    }
    prev = 1.0;
    rises = 0;
  }
  // returns status if the iteration must stop
  int push(double rel, int cycles, int refinements, double tol, int max_cycles) {
    if (info) {
      if (info->n_hist < CSFF_MAX_HISTORY) info->history[info->n_hist++] = rel;
      info->cycles = cycles;
      info->refinements = refinements;
      info->rel_res = rel;
      info->conv_factor = cycles > 0 ? std::pow(rel, 1.0 / cycles) : 0.0;
    }
    if (!std::isfinite(rel)) return CSFF_ERR_NONFINITE;
    if (rel <= tol) return CSFF_OK;
    rises = rel > prev ? rises + 1 : 0;
    prev = rel;
    if (rises >= 3) return CSFF_ERR_DIVERGED;
    if (cycles >= max_cycles) return CSFF_ERR_NOT_CONVERGED;
    return -1;
  }
};

// V-cycle from level l0 (u, b: that level's iterate and right-hand side) with
// the fused 2D V(1,1) RB-GS kernels down to the coarse-level block.
template <typename T>
csff_status run_fused_from(csff_plan* P, int l0, cx<T>* u, const cx<T>* b, bool zero_init) {
  cudaStream_t s = P->stream;
  const int lc = P->fused_lc;
  for (int l = l0; l < lc; ++l) {
    Level& F = P->lv[l];
    Level& C = P->lv[l + 1];
    const cx<T>* in = (l == l0) ? u : ubuf<T>(F);
    const cx<T>* bl = (l == l0) ? b : bbuf<T>(F);
    CK(csff::launch_down2<T>(F, C, in, zero_init || l > l0, bl, tbuf<T>(F), bbuf<T>(C), s, l == 0), "fused down");
  }
  CK(csff::launch_coarse_levels<T>(P->dim, P->lv, lc, cinv<T>(P), coarse_fp64(P) ? P->coarse_inv : nullptr,
                                   bbuf<T>(P->lv[lc]), ubuf<T>(P->lv[lc]), s),
     "coarse levels");
  for (int l = lc - 1; l >= l0; --l) {
    Level& F = P->lv[l];
    Level& C = P->lv[l + 1];
    cx<T>* out = (l == l0) ? u : ubuf<T>(F);
    const cx<T>* bl = (l == l0) ? b : bbuf<T>(F);
    CK(csff::launch_up2<T>(F, C, tbuf<T>(F), ubuf<T>(C), bl, out, s, l == 0), "fused up");
  }
  return CSFF_OK;
}

// With the learned step active: levels below learned_levels run the per-level
// kernels (red-black sweep, learned step, residual, full weighting; then
// prolongation, sweep, learned step), the levels below them the fused kernels.
csff_status run_vcycle_learned(csff_plan* P, float2* u, const float2* b, bool zero_init) {
  cudaStream_t s = P->stream;
  const int ll = P->learned_levels;
  for (int l = 0; l < ll; ++l) {
    Level& L = P->lv[l];
    Level& C = P->lv[l + 1];
    float2* ul = (l == 0) ? u : L.u32;
    const float2* bl = (l == 0) ? b : L.b32;
    if (l > 0 || zero_init) CK(csff::launch_zero<float>(ul, L.N, s), "zero");
    CS(smooth<float>(P, l, ul, bl, 1));
    CK(csff::launch_residual<float>(P->dim, L, ul, bl, L.r32, s), "residual");
    CK(csff::launch_restrict<float>(P->dim, L, C, L.r32, C.b32, s), "restrict");
  }
  CS(run_fused_from<float>(P, ll, P->lv[ll].u32, P->lv[ll].b32, true));
  for (int l = ll - 1; l >= 0; --l) {
    Level& L = P->lv[l];
    Level& C = P->lv[l + 1];
    float2* ul = (l == 0) ? u : L.u32;
    const float2* bl = (l == 0) ? b : L.b32;
    CK(csff::launch_prolong_add<float>(P->dim, L, C, C.u32, ul, s), "prolong");
    CS(smooth<float>(P, l, ul, bl, 1));
  }
  return CSFF_OK;
}

// One V-cycle at the finest level: the fused 2D V(1,1) RB-GS kernels when the
// plan qualifies, else the general per-step kernels.  zero_init: the iterate
// enters as zero (the correction equation of a refinement step).
template <typename T>
csff_status run_vcycle(csff_plan* P, cx<T>* u, const cx<T>* b, bool zero_init) {
  const int lc = P->fused_lc;
  if constexpr (sizeof(T) == 4) {
    if (P->net && !P->learned_off) {
      if (lc > P->learned_levels) return run_vcycle_learned(P, u, b, zero_init);
      if (zero_init) CK(csff::launch_zero<T>(u, P->lv[0].N, P->stream), "zero");
      return vcycle<T>(P, 0, u, b);
    }
  }
  if (lc < 1) {
    if (zero_init) CK(csff::launch_zero<T>(u, P->lv[0].N, P->stream), "zero");
    return vcycle<T>(P, 0, u, b);
  }
  return run_fused_from<T>(P, 0, u, b, zero_init);
}

// Body of one solver step on P->stream (eagerly or under capture): the
// finest-level norm of the new residual ends in red_host[0].
csff_status step_fp64(csff_plan* P, int eb) {
  Level& L = P->lv[0];
  CS(run_vcycle<double>(P, L.u64, L.b64, false));
  CK(csff::launch_residual<double>(P->dim, L, L.u64, L.b64, L.r64, P->stream), "residual");
  CS(norm64(P, L.r64, eb, 0));
  CK(cudaMemcpyAsync(P->red_host, P->red_out, sizeof(double), cudaMemcpyDeviceToHost, P->stream), "read norm");
  return CSFF_OK;
}

// One refinement step of the mixed solve: n FP32 V-cycles on A e = r' (r' the
// scaled residual, already the FP32 right-hand side), u' += e, the new r' in
// double-float and its norm (refine_df.cu)
csff_status step_mixed(csff_plan* P, int n) {
  Level& L = P->lv[0];
  cudaStream_t s = P->stream;
  for (int c = 0; c < n; ++c) CS(run_vcycle<float>(P, L.u32, L.b32, c == 0));
  CK(csff::launch_df_update(P->dfu, L.u32, L.N, s), "update");
  CK(csff::launch_df_residual(P->dim, L, P->dfu, P->dfb, P->dfq, L.b32, P->dfpart, P->red_out, s), "residual");
  CK(cudaMemcpyAsync(P->red_host, P->red_out, sizeof(double), cudaMemcpyDeviceToHost, s), "read norm");
  return CSFF_OK;
}

void destroy_graphs(csff_plan* P) {
  for (auto& g : P->graphs)
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
}

// One refinement step with the FP64 residual and update (option refine_fp64):
// n FP32 V-cycles on A e = r32 (r32 = 2^-e_b r, already in the cycles'
// right-hand side), u += 2^e_b e in FP64, then in one pass the new FP64
// residual, its FP32 rounding 2^-e_b r as the next right-hand side and its norm
// (e_b the exponent of max |b|, fixed for the solve)
csff_status step_mixed64(csff_plan* P, int n) {
  Level& L = P->lv[0];
  cudaStream_t s = P->stream;
  for (int c = 0; c < n; ++c) CS(run_vcycle<float>(P, L.u32, L.b32, c == 0));
  CK(csff::launch_update64_fixed(L.u64, L.u32, L.N, P->refine_eb, s), "update");
  CK(csff::launch_refine_residual(P->dim, L, L.u64, L.b64, P->refine_eb, L.b32, P->red, P->red_blocks, P->red_out,
                                  s),
     "residual");
  CK(cudaMemcpyAsync(P->red_host, P->red_out, sizeof(double), cudaMemcpyDeviceToHost, s), "read norm");
  return CSFF_OK;
}

// Run one step: replay the captured graph (capturing it first if the key
// changed), or eagerly while kernel families of the solver are being timed.
// arg: the body's parameter (FP64 step: the right-hand side's exponent; mixed
// step: its FP32 cycle count), part of what the key identifies.
csff_status run_step(csff_plan* P, long long key, csff_status (*body)(csff_plan*, int), int arg) {
  const unsigned mg_bits = CSFF_PROF_MG32 | CSFF_PROF_MG64 | CSFF_PROF_TILES32 | CSFF_PROF_TILES32_FINE;
  if (!P->use_graphs || !P->gstream || (csff::prof_mask() & mg_bits)) {
    CS(body(P, arg));
    CK(cudaStreamSynchronize(P->stream), "sync");
    return CSFF_OK;
  }
  csff_plan::StepGraph* G = nullptr;
  for (auto& g : P->graphs)
    if (g.exec && g.key == key) G = &g;
  if (!G) {
    G = &P->graphs[P->graph_next];
    P->graph_next = (P->graph_next + 1) % csff_plan::GRAPH_SLOTS;
    if (G->exec) { cudaGraphExecDestroy(G->exec); G->exec = nullptr; }
    CK(cudaStreamBeginCapture(P->gstream, cudaStreamCaptureModeThreadLocal), "begin capture");
    const uint64_t before = csff::g_launches.load();
    cudaStream_t saved = P->stream;
    P->stream = P->gstream;
    csff::g_capturing = true;
    csff_status st = body(P, arg);
    csff::g_capturing = false;
    P->stream = saved;
    // kernels recorded in the graph: counted again on every replay below
    G->kernels = csff::g_launches.load() - before;
    csff::g_launches.fetch_sub(G->kernels);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(P->gstream, &graph);
    if (st != CSFF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return csff::cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&G->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { G->exec = nullptr; return csff::cuda_fail(e, "instantiate graph"); }
    G->key = key;
  }
  CK(cudaEventRecord(P->gev, P->stream), "event");
  CK(cudaStreamWaitEvent(P->gstream, P->gev, 0), "wait event");
  CK(cudaGraphLaunch(G->exec, P->gstream), "graph launch");
  csff::count_launch((int)G->kernels);
  CK(cudaStreamSynchronize(P->gstream), "sync");
  return CSFF_OK;
}

// One FP64 V-cycle on level l of the full-multigrid iteration (iterate and
// right-hand side in that level's u64 and b64; the levels below serve as the
// cycle's work space), then the level's residual norm into red_host[0].  The
// level travels in the step argument: l * 8192 + (e + 4096), e the prescale
// exponent of the norms.
csff_status step_fmg_level(csff_plan* P, int arg) {
  const int l = arg / 8192, e = arg % 8192 - 4096;
  Level& L = P->lv[l];
  if (P->fused_lc > l) CS(run_fused_from<double>(P, l, L.u64, L.b64, false));
  else CS(vcycle<double>(P, l, L.u64, L.b64));
  CK(csff::launch_residual<double>(P->dim, L, L.u64, L.b64, L.r64, P->stream), "residual");
  CK(csff::launch_norm2<double>(L.r64, L.N, e, P->red, P->red_blocks, P->red_out, P->stream), "norm");
  CK(cudaMemcpyAsync(P->red_host, P->red_out, sizeof(double), cudaMemcpyDeviceToHost, P->stream), "read norm");
  return CSFF_OK;
}

// FP64 V-cycles on the finest level (iterate in the plan's u64, rhs in b64).
csff_status solve_fp64(csff_plan* P, int eb, double nb, csff_info* info) {
  Tracker tr;
  tr.start(info);
  int cycles = 0;
  const long long key = (1ll << 40) + (long long)(eb + 8192);
  for (;;) {
    CS(run_step(P, key, step_fp64, eb));
    ++cycles;
    int st = tr.push(P->red_host[0] / nb, cycles, 0, P->opts.rel_tol, P->opts.max_cycles);
    if (st >= 0) return (csff_status)st;
  }
}

// Mixed solve: FP32 V-cycles on the correction equation inside a refinement whose
// residual and update run in double-float arithmetic (refine_df.cu).  guess: the
// initial iterate (nullptr: zero); the solution is written to u_out (which may be
// the guess's buffer).
csff_status solve_mixed(csff_plan* P, int eb, double nb, csff_info* info, const double2* guess, double2* u_out) {
  Level& L = P->lv[0];
  Tracker tr;
  tr.start(info);
  int cycles = 0, refinements = 0;
  const int inner = P->opts.inner_cycles > 0 ? P->opts.inner_cycles : 1;
  const bool r64 = P->opts.refine_fp64 != 0;
  // the step's graph depends on its cycle count, on whether the learned step
  // runs and, with the FP64 refinement, on the right-hand side's exponent (the
  // prescale of its norm)
  const long long key0 = r64 ? (3ll << 40) + (long long)(eb + 8192) * 4096 : 2ll << 40;
  const bool adaptive = P->opts.adaptive_inner != 0;
  int n = inner;
  // with a learned smoother the first two refinement steps run plain
  // red-black sweeps and the second sets the reference factor; a later learned
  // step that reduces the residual less than min(reference, guard) hands the
  // rest of the solve back to plain sweeps
  P->learned_off = P->net != nullptr;
  bool fell_back = false;
  double prev = 1.0, ref_factor = P->learned_guard;
  // double-float: b' = 2^-eb b and q are split already (solve_loaded); u' =
  // 2^-eb u (guess or zero).  FP64: u in L.u64, its residual and norm.
  cudaStream_t s = P->stream;
  if (r64) {
    // the first right-hand side of the FP32 cycles: 2^-eb r for the guess, or
    // 2^-eb b from zero
    P->refine_eb = eb;
    if (guess) {
      CK(cudaMemcpyAsync(L.u64, guess, sizeof(double2) * (size_t)L.N, cudaMemcpyDeviceToDevice, s), "copy guess");
      CK(csff::launch_refine_residual(P->dim, L, L.u64, L.b64, eb, L.b32, P->red, P->red_blocks, P->red_out, s),
         "residual");
    } else {
      CK(csff::launch_zero<double>(L.u64, L.N, s), "zero");
      CK(csff::launch_scale_to32(L.b64, L.N, eb, L.b32, s), "scale b");
    }
  } else if (guess) {
    CK(csff::launch_df_split(guess, L.N, -eb, P->dfu, nullptr, nullptr, nullptr, s), "split u");
    CK(csff::launch_df_residual(P->dim, L, P->dfu, P->dfb, P->dfq, L.b32, nullptr, nullptr, s), "residual");
  } else {
    // u' = 0: the first residual is b' itself, already in L.b32 (rounded to FP32
    // by the split)
    CK(cudaMemsetAsync(P->dfu, 0, sizeof(float4) * (size_t)L.N, s), "zero u");
  }
  const double nbs = r64 ? nb : std::ldexp(nb, -eb);   // ||b|| or ||b'||, the norms' scale
  csff_status result = CSFF_OK;
  for (;;) {
    const bool learned = P->net && !P->learned_off;
    const int n_step = n;
    const double rel_before = prev;
    CS(run_step(P, key0 + n_step + (learned ? (1ll << 38) : 0), r64 ? step_mixed64 : step_mixed, n_step));
    cycles += n_step;
    ++refinements;
    const double rel = P->red_host[0] / nbs;
    // the learned step's comparisons use the reduction of a step of inner
    // cycles (steps of the adaptive schedule differ in length)
    const double factor = n_step == inner ? rel / prev : std::pow(rel / prev, (double)inner / n_step);
    if (P->net && refinements <= 2) {
      // two plain steps: the second one's factor is the reference
      if (refinements == 2) {
        ref_factor = std::min(factor, P->learned_guard);
        P->learned_off = false;
      }
    } else if (learned && factor > ref_factor) {
      P->learned_off = true;
      fell_back = true;
    }
    prev = rel;
    int st = tr.push(rel, cycles, refinements, P->opts.rel_tol, P->opts.max_cycles);
    if (info) info->flags = (P->net ? 1 : 0) | (fell_back ? 2 : 0);
    if (st >= 0) {
      result = (csff_status)st;
      break;
    }
    // adaptive: the next step runs the cycles that this step's per-cycle factor
    // rho predicts for rel rho^n <= rel_tol (a guess makes the first step's
    // starting residual unknown, so adapting starts after the second step)
    n = inner;
    if (adaptive && (!guess || refinements >= 2))
      n = csff_refinement_cycles(rel_before, rel, n_step, P->opts.rel_tol, inner);
  }
  if (r64)
    CK(cudaMemcpyAsync(u_out, L.u64, sizeof(double2) * (size_t)L.N, cudaMemcpyDeviceToDevice, s), "copy");
  else
    CK(csff::launch_df_to64(P->dfu, L.N, eb, u_out, s), "assemble u");     // u = 2^eb (hi + lo)
  return result;
}

csff_status check_level(const csff_plan* P, int level, int arith) {
  if (!P) return invalid("plan is NULL");
  if (level < 0 || level >= (int)P->lv.size()) return invalid("level out of range");
  if (arith != CSFF_ARITH_FP64 && arith != CSFF_ARITH_FP32) return invalid("arith must be FP64 or FP32");
  return CSFF_OK;
}

int worse(int a, int b) {
  auto rank = [](int s) { return s == CSFF_OK ? 0 : (s == CSFF_WARN_ILL_CONDITIONED ? 1 : 2 + s); };
  return rank(b) > rank(a) ? b : a;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

double csff_gamma_from_ecs(double theta) { return std::atan(std::sin(theta) / (2.0 + std::cos(theta))); }

int csff_refinement_cycles(double rel_before, double rel_after, int cycles_run, double rel_tol, int max_cycles) {
  return csff::refinement_cycles(rel_before, rel_after, cycles_run, rel_tol, max_cycles);
}

const char* csff_status_string(csff_status s) {
  switch (s) {
    case CSFF_OK: return "ok";
    case CSFF_ERR_INVALID_ARG: return "invalid argument";
    case CSFF_ERR_CUDA: return "CUDA error";
    case CSFF_ERR_OOM: return "out of device memory";
    case CSFF_ERR_NOT_CONVERGED: return "not converged";
    case CSFF_ERR_DIVERGED: return "diverged";
    case CSFF_ERR_NONFINITE: return "non-finite value";
    case CSFF_ERR_TIMEOUT: return "device wait timed out";
    case CSFF_ERR_UNSUPPORTED: return "unsupported";
    case CSFF_WARN_ILL_CONDITIONED: return "ill-conditioned (result valid)";
  }
  return "unknown status";
}

const char* csff_last_error(void) { return csff::t_last_error.c_str(); }

uint64_t csff_kernel_launches(void) { return csff::g_launches.load(); }

csff_status csff_prof_begin(unsigned family_mask) {
  for (auto& r : csff::g_prof.recs) {
    csff::g_prof.pool.push_back(r.a);
    csff::g_prof.pool.push_back(r.b);
  }
  csff::g_prof.recs.clear();
  csff::g_prof.mask = family_mask;
  return CSFF_OK;
}

csff_status csff_prof_end(csff_prof_stats* out) {
  if (!out) return invalid("NULL output");
  csff::g_prof.mask = 0;
  std::memset(out, 0, sizeof(csff_prof_stats) * CSFF_PROF_FAMILIES);
  for (auto& r : csff::g_prof.recs) {
    CK(cudaEventSynchronize(r.b), "profiling event");
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, r.a, r.b), "profiling elapsed time");
    csff_prof_stats& o = out[r.family];
    o.launches += 1;
    o.ms += ms;
    o.alg_bytes += r.bytes;
    o.alg_flops += r.flops;
  }
  return CSFF_OK;
}

void csff_plan_destroy(csff_plan* P) {
  if (!P) return;
  for (Level& L : P->lv)
    for (void* p : {(void*)L.q64, (void*)L.dinv64, (void*)L.q32, (void*)L.dinv32, (void*)L.u64, (void*)L.t64,
                    (void*)L.b64, (void*)L.r64, (void*)L.u32, (void*)L.t32, (void*)L.b32, (void*)L.r32,
                    (void*)L.fac32})
      if (p) cudaFree(p);
  for (double2* p : P->chi_tab)
    if (p) cudaFree(p);
  if (P->coarse_inv) cudaFree(P->coarse_inv);
  if (P->coarse_inv32) cudaFree(P->coarse_inv32);
  if (P->uinc_tab) cudaFree(P->uinc_tab);
  if (P->red) cudaFree(P->red);
  if (P->red_out) cudaFree(P->red_out);
  if (P->red_host) cudaFreeHost(P->red_host);
  for (void* p : {P->gm_v, (void*)P->gm_part, (void*)P->gm, (void*)P->sep_T, (void*)P->dfu, (void*)P->dfb,
                  (void*)P->dfq, (void*)P->dfpart})
    if (p) cudaFree(p);
  csff::free_ff_buffers(P);
  destroy_graphs(P);
  if (P->gstream) cudaStreamDestroy(P->gstream);
  if (P->gev) cudaEventDestroy(P->gev);
  delete P;
}

csff_status csff_plan_create(const csff_problem* prob, const csff_opts* opts, void* stream, csff_plan** out) {
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  if (!prob || !opts) return invalid("problem/opts is NULL");
  if (prob->dim != 2 && prob->dim != 3) return invalid("dim must be 2 or 3");
  if (!(prob->gamma > 0.0 && prob->gamma < 0.78539816339744830962)) return invalid("gamma must lie in (0, pi/4)");
  if (!(prob->k > 0.0) || !std::isfinite(prob->k)) return invalid("k must be positive");
  if (!(prob->box_hi > prob->box_lo)) return invalid("empty box");
  if (prob->n_gauss < 0 || prob->n_gauss > 8 || (prob->n_gauss > 0 && !prob->gauss))
    return invalid("n_gauss must be 0..8 with a non-NULL array");
  for (int g = 0; g < prob->n_gauss; ++g)
    if (!(prob->gauss[g].width > 0.0)) return invalid("Gaussian width must be positive");
  if (opts->smoother != CSFF_SMOOTHER_JACOBI && opts->smoother != CSFF_SMOOTHER_RBGS &&
      opts->smoother != CSFF_SMOOTHER_GMRES)
    return invalid("unknown smoother");
  if (opts->smoother == CSFF_SMOOTHER_GMRES && (opts->krylov_m < 0 || opts->krylov_m > csff::GM_MAX))
    return invalid("krylov_m must be 0..4 (0 selects 3)");
  if (opts->adaptive_inner != 0 && opts->adaptive_inner != 1) return invalid("adaptive_inner must be 0 or 1");
  if (opts->refine_fp64 != 0 && opts->refine_fp64 != 1) return invalid("refine_fp64 must be 0 or 1");
  if (opts->nu1 < 0 || opts->nu2 < 0 || opts->nu1 + opts->nu2 == 0) return invalid("need nu1 + nu2 > 0");
  if (opts->precision != CSFF_PREC_FP64 && opts->precision != CSFF_PREC_MIXED) return invalid("bad precision");
  if (!(opts->rel_tol > 0.0) || opts->max_cycles < 1) return invalid("need rel_tol > 0 and max_cycles >= 1");
  if (opts->smoother == CSFF_SMOOTHER_JACOBI && !(opts->omega > 0.0 && opts->omega < 2.0))
    return invalid("omega must lie in (0, 2)");
  if (opts->coarsest_n < 3) return invalid("coarsest_n must be >= 3");
  std::vector<int> ns;
  for (int n = prob->n;; n = (n + 1) / 2) {
    ns.push_back(n);
    if (n == opts->coarsest_n) break;
    if (n < opts->coarsest_n || (n - 1) % 2 != 0 || ns.size() > 15)
      return invalid("n must equal 2^j (coarsest_n - 1) + 1 with at most 16 levels");
  }
  const int d = prob->dim;
  long long nc = 1;
  for (int i = 0; i < d; ++i) nc *= (opts->coarsest_n - 2);
  if (nc > 4096) return invalid("coarsest grid too large for the dense direct solve");

  csff_plan* P = new csff_plan();
  P->prob = *prob;
  P->gauss.assign(prob->gauss, prob->gauss + prob->n_gauss);
  P->prob.gauss = P->gauss.data();
  P->opts = *opts;
  if (P->opts.smoother == CSFF_SMOOTHER_GMRES && P->opts.krylov_m == 0) P->opts.krylov_m = 3;
  P->dim = d;
  P->stream = (cudaStream_t)stream;
  auto fail = [&](csff_status s) {
    csff_plan_destroy(P);
    return s;
  };
  const double k2 = prob->k * prob->k;
  const std::complex<double> e2 = std::polar(1.0, -2.0 * prob->gamma);
  for (size_t l = 0; l < ns.size(); ++l) {
    Level L;
    L.n = ns[l];
    L.m = L.n - 2;
    L.N = 1;
    for (int i = 0; i < d; ++i) L.N *= L.m;
    L.h = (prob->box_hi - prob->box_lo) / (L.n - 1);
    std::complex<double> c = e2 / (L.h * L.h);
    L.c = make_double2(c.real(), c.imag());
    P->lv.push_back(L);
  }
  for (size_t l = 0; l < P->lv.size(); ++l) {
    Level& L = P->lv[l];
    csff_status s;
    if ((s = dev_alloc(P, &L.q64, L.N)) || (s = dev_alloc(P, &L.dinv64, L.N)) || (s = dev_alloc(P, &L.q32, L.N)) ||
        (s = dev_alloc(P, &L.dinv32, L.N)) || (s = dev_alloc(P, &L.u64, L.N)) || (s = dev_alloc(P, &L.t64, L.N)) ||
        (s = dev_alloc(P, &L.b64, L.N)) || (s = dev_alloc(P, &L.r64, L.N)) || (s = dev_alloc(P, &L.u32, L.N)) ||
        (s = dev_alloc(P, &L.t32, L.N)) || (s = dev_alloc(P, &L.b32, L.N)) || (s = dev_alloc(P, &L.r32, L.N)))
      return fail(s);
    std::vector<double2> tab = chi_tables(P, L.n);
    double2* dtab = nullptr;
    if ((s = dev_alloc(P, &dtab, tab.size()))) return fail(s);
    P->chi_tab.push_back(dtab);
    cudaError_t e = cudaMemcpy(dtab, tab.data(), sizeof(double2) * tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(csff::cuda_fail(e, "upload chi tables"));
    if (d == 2) {
      std::vector<float2> fac = fp32_factors(P, tab, L.m);
      L.ng = P->prob.n_gauss;
      L.k2 = P->prob.k * P->prob.k;
      if (!fac.empty()) {
        if ((s = dev_alloc(P, &L.fac32, fac.size()))) return fail(s);
        e = cudaMemcpy(L.fac32, fac.data(), sizeof(float2) * fac.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(csff::cuda_fail(e, "upload factors"));
      }
    }
    std::vector<const double2*> per_g(P->prob.n_gauss);
    for (int g = 0; g < P->prob.n_gauss; ++g) per_g[g] = dtab + (size_t)g * d * L.m;
    e = csff::launch_coefs(d, L, per_g.data(), P->prob.n_gauss, k2, P->stream);
    if (e != cudaSuccess) return fail(csff::cuda_fail(e, "coefficients"));
  }
  // the chi tables are kept per level; finest-level tables are used by rhs/far field
  std::vector<double2> inv;
  if (!coarse_inverse(P, P->lv.back(), inv)) return fail(invalid("coarsest operator is singular"));
  P->coarse_N = (int)std::lround(std::sqrt((double)inv.size()));
  {
    csff_status s;
    std::vector<float2> inv32(inv.size());
    for (size_t i = 0; i < inv.size(); ++i) inv32[i] = make_float2((float)inv[i].x, (float)inv[i].y);
    if ((s = dev_alloc(P, &P->coarse_inv, inv.size())) || (s = dev_alloc(P, &P->coarse_inv32, inv.size())))
      return fail(s);
    cudaError_t e = cudaMemcpy(P->coarse_inv, inv.data(), sizeof(double2) * inv.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(P->coarse_inv32, inv32.data(), sizeof(float2) * inv32.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(csff::cuda_fail(e, "upload coarse inverse"));
    P->red_blocks = 152 * 8;
    if ((s = dev_alloc(P, &P->red, P->red_blocks)) || (s = dev_alloc(P, &P->red_out, 16)) ||
        (s = dev_alloc(P, &P->uinc_tab, (size_t)d * P->lv[0].m)))
      return fail(s);
    e = cudaMallocHost((void**)&P->red_host, 16 * sizeof(double));
    if (e != cudaSuccess) return fail(csff::cuda_fail(e, "pinned host buffer"));
    if (P->opts.precision == CSFF_PREC_MIXED &&
        ((s = dev_alloc(P, &P->dfu, (size_t)P->lv[0].N)) || (s = dev_alloc(P, &P->dfb, (size_t)P->lv[0].N)) ||
         (s = dev_alloc(P, &P->dfq, (size_t)P->lv[0].N)) ||
         (s = dev_alloc(P, &P->dfpart, (size_t)std::max(csff::df_residual_blocks(d, P->lv[0].m),
                                                         csff::df_split_blocks(P->lv[0].N))))))
      return fail(s);
    if (P->opts.smoother == CSFF_SMOOTHER_GMRES) {
      double2* v = nullptr;
      if ((s = dev_alloc(P, &v, (size_t)(P->opts.krylov_m + 1) * P->lv[0].N)) ||
          (s = dev_alloc(P, &P->gm_part, P->red_blocks)) || (s = dev_alloc(P, &P->gm, 1))) {
        if (v) cudaFree(v);
        return fail(s);
      }
      P->gm_v = v;
    }
  }
  // fused V(1,1) RB-GS path (2D): the levels from the first with n <= 33 run in
  // one CTA; at least one fused fine level is needed
  if (d == 2 && opts->smoother == CSFF_SMOOTHER_RBGS && opts->nu1 == 1 && opts->nu2 == 1) {
    int lc = -1;
    for (int l = 0; l < (int)P->lv.size(); ++l)
      if (P->lv[l].n <= 33) { lc = l; break; }
    if (lc < 0) lc = (int)P->lv.size() - 1;
    if (lc >= 1 && csff::coarse_levels_smem(d, P->lv, lc, 8) <= 200 * 1024) {
      cudaError_t e = csff::prepare_fused(d, P->lv, lc);
      if (e != cudaSuccess) return fail(csff::cuda_fail(e, "fused kernel attributes"));
      P->fused_lc = lc;
    }
  }
  {
    cudaError_t e = cudaStreamCreateWithFlags(&P->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->gev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(csff::cuda_fail(e, "graph stream"));
  }
  // conditioning estimates (single Gaussian on the axis of eta, Sec. 3.3's
  // warning about products of growing and decaying factors)
  {
    const double sg = std::sin(prob->gamma), c2 = std::cos(2 * prob->gamma);
    const double R = std::max(std::fabs(prob->box_lo), std::fabs(prob->box_hi));
    double lr = -1e300, lf = -1e300;
    for (int g = 0; g < prob->n_gauss; ++g) {
      double w = prob->gauss[g].width, la = std::log(std::hypot(prob->gauss[g].amp_re, prob->gauss[g].amp_im));
      double t = std::min(prob->k * sg * w / (2 * c2), R);
      lr = std::max(lr, la + prob->k * sg * t - c2 * t * t / w);
      double t2 = std::min(prob->k * sg * w / c2, R);
      lf = std::max(lf, la + 2 * prob->k * sg * t2 - c2 * t2 * t2 / w);
    }
    P->log_rhs_max = lr;
    P->log_ff_max = lf;
  }
  cudaError_t e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return fail(csff::cuda_fail(e, "plan setup"));
  *out = P;
  return CSFF_OK;
}

csff_status csff_plan_set_learned(csff_plan* P, csff_net* net, int levels, double guard) {
  if (!P) return invalid("plan is NULL");
  if (net && (levels < 1 || levels > (int)P->lv.size() - 1 || !(guard > 0.0))) return invalid("bad learned settings");
  if (net && P->opts.smoother != CSFF_SMOOTHER_RBGS) {
    csff::set_error("the learned step follows red-black sweeps");
    return CSFF_ERR_UNSUPPORTED;
  }
  if (net && csff::net_dim(net) != P->dim) return invalid("the network's dimension is not the plan's");
  if (net) CS(csff::net_reserve(net, P->lv[0].N));
  P->net = net;
  P->learned_levels = net ? levels : 0;
  P->learned_guard = guard;
  for (auto& n : P->level_net) n = nullptr;
  destroy_graphs(P);
  return CSFF_OK;
}

csff_status csff_plan_set_learned_level(csff_plan* P, int level, csff_net* net) {
  if (!P) return invalid("plan is NULL");
  if (!P->net || level < 0 || level >= P->learned_levels) return invalid("level carries no learned step");
  if (net && csff::net_dim(net) != P->dim) return invalid("the network's dimension is not the plan's");
  if (net) CS(csff::net_reserve(net, P->lv[level].N));
  P->level_net[level] = net;
  destroy_graphs(P);
  return CSFF_OK;
}

csff_status csff_plan_copy_coefficients(const csff_plan* P, int level, void* q32_dev, double* c_host) {
  if (!P || level < 0 || level >= (int)P->lv.size() || !q32_dev || !c_host) return invalid("bad arguments");
  const Level& L = P->lv[level];
  CK(cudaMemcpyAsync(q32_dev, L.q32, sizeof(float2) * (size_t)L.N, cudaMemcpyDeviceToDevice, P->stream), "copy q");
  CK(cudaStreamSynchronize(P->stream), "sync");
  c_host[0] = L.c.x;
  c_host[1] = L.c.y;
  return CSFF_OK;
}

csff_status csff_plan_set_stream(csff_plan* P, void* stream) {
  if (!P) return invalid("plan is NULL");
  P->stream = (cudaStream_t)stream;
  return CSFF_OK;
}

csff_status csff_plan_describe(const csff_plan* P, csff_plan_desc* d) {
  if (!P || !d) return invalid("NULL argument");
  std::memset(d, 0, sizeof(*d));
  d->n_levels = (int)P->lv.size();
  for (int l = 0; l < d->n_levels; ++l) {
    d->n[l] = P->lv[l].n;
    d->h[l] = P->lv[l].h;
  }
  d->device_bytes = P->bytes;
  d->log_rhs_max = P->log_rhs_max;
  d->log_ff_max = P->log_ff_max;
  d->ill_conditioned = P->log_ff_max > 600.0;
  d->below_min_gamma = P->prob.gamma < std::atan(0.5) / 2.0;
  return CSFF_OK;
}

csff_status csff_rhs(csff_plan* P, int n_rhs, const double* eta, void* b_dev) {
  if (!P || !eta || !b_dev || n_rhs < 0) return invalid("bad rhs arguments");
  Level& L = P->lv[0];
  std::vector<const double2*> per_g(P->prob.n_gauss);
  for (int g = 0; g < P->prob.n_gauss; ++g) per_g[g] = P->chi_tab[0] + (size_t)g * P->dim * L.m;
  for (int r = 0; r < n_rhs; ++r) {
    CS(upload_uinc(P, eta + (size_t)r * P->dim));
    CK(csff::launch_rhs(P->dim, L.m, per_g.data(), P->prob.n_gauss, P->uinc_tab, P->prob.k * P->prob.k,
                        (double2*)b_dev + (size_t)r * L.N, P->stream),
       "rhs");
  }
  return CSFF_OK;
}

static csff_status solve_loaded(csff_plan* P, double2* u, int use_guess, csff_info* in);

csff_status csff_solve(csff_plan* P, int n_rhs, const double* eta, void* u_dev, int use_guess, csff_info* info) {
  if (!P || !eta || !u_dev || n_rhs < 0) return invalid("bad solve arguments");
  Level& L = P->lv[0];
  int worst = CSFF_OK;
  for (int r = 0; r < n_rhs; ++r) {
    double2* u = (double2*)u_dev + (size_t)r * L.N;
    csff_info* in = info ? info + r : nullptr;
    CS(csff_rhs(P, 1, eta + (size_t)r * P->dim, L.b64));
    const csff_status st = solve_loaded(P, u, use_guess, in);
    if (st == CSFF_ERR_CUDA || st == CSFF_ERR_OOM || st == CSFF_ERR_INVALID_ARG) return st;
    worst = worse(worst, st);
  }
  return (csff_status)worst;
}

// Solve A u = b for the right-hand side already in level 0's b64; u (the
// caller's buffer) holds the guess when use_guess and receives the solution.
// Full multigrid (Sec. 4, FMG paragraph; Table 3) for the right-hand side in
// level 0's b64: b_{l+1} = FW(b_l) down to the coarsest level, its direct
// solve, then on each finer level the interpolated coarser solution as the
// initial guess of FP64 V-cycles to rel_tol ||b_l||.
static csff_status fmg_loaded(csff_plan* P, double2* u_out, int* level_cycles, csff_info* in) {
  const int nl = (int)P->lv.size();
  cudaStream_t s = P->stream;
  Level& L0 = P->lv[0];
  int* ex = reinterpret_cast<int*>(P->red_out + 4);
  CK(csff::launch_max_exp(L0.b64, L0.N, ex, s), "max exponent");
  int eb = 0;
  CK(cudaMemcpyAsync(&eb, ex, sizeof(int), cudaMemcpyDeviceToHost, s), "read exponent");
  CK(cudaStreamSynchronize(s), "sync");
  if (in) { std::memset(in, 0, sizeof(*in)); in->n_hist = 1; }
  if (eb >= 4000) {
    csff::set_error("right-hand side is not finite");
    if (in) in->status = CSFF_ERR_NONFINITE;
    return CSFF_ERR_NONFINITE;
  }
  if (eb <= -2000) eb = 0;
  for (int l = 1; l < nl; ++l)
    CK(csff::launch_restrict<double>(P->dim, P->lv[l - 1], P->lv[l], P->lv[l - 1].b64, P->lv[l].b64, s), "restrict");
  CK(csff::launch_coarse_solve<double>(P->coarse_inv, P->coarse_N, P->lv[nl - 1].b64, P->lv[nl - 1].u64, s),
     "coarse solve");
  csff_status result = CSFF_OK;
  for (int l = nl - 2; l >= 0; --l) {
    Level& L = P->lv[l];
    CK(csff::launch_zero<double>(L.u64, L.N, s), "zero");
    CK(csff::launch_prolong_add<double>(P->dim, L, P->lv[l + 1], P->lv[l + 1].u64, L.u64, s), "interpolate");
    CK(csff::launch_norm2<double>(L.b64, L.N, eb, P->red, P->red_blocks, P->red_out + 1, s), "norm b");
    CK(csff::launch_residual<double>(P->dim, L, L.u64, L.b64, L.r64, s), "residual");
    CK(csff::launch_norm2<double>(L.r64, L.N, eb, P->red, P->red_blocks, P->red_out, s), "norm");
    CS(read_scalars(P, 2));
    const double nb = P->red_host[1];
    int cycles = 0;
    csff_status st = CSFF_OK;
    if (nb > 0.0) {
      Tracker tr;
      tr.start(l == 0 ? in : nullptr);
      double rel = P->red_host[0] / nb;
      if (l == 0 && in) in->history[0] = rel;
      tr.prev = rel;
      if (rel > P->opts.rel_tol) {
        const long long key = (5ll << 40) + (long long)l * 8192 + (eb + 4096);
        for (;;) {
          CS(run_step(P, key, step_fmg_level, l * 8192 + (eb + 4096)));
          ++cycles;
          rel = P->red_host[0] / nb;
          const int t = tr.push(rel, cycles, 0, P->opts.rel_tol, P->opts.max_cycles);
          if (t >= 0) { st = (csff_status)t; break; }
        }
      } else if (l == 0 && in) {
        in->rel_res = rel;
      }
    }
    if (level_cycles) level_cycles[nl - 2 - l] = cycles;
    result = (csff_status)worse(result, st);
  }
  CK(cudaMemcpyAsync(u_out, L0.u64, sizeof(double2) * (size_t)L0.N, cudaMemcpyDeviceToDevice, s), "copy");
  if (in) in->status = result;
  return result;
}

static csff_status solve_loaded(csff_plan* P, double2* u, int use_guess, csff_info* in) {
  Level& L = P->lv[0];
  if (!use_guess) CK(csff::launch_zero<double>(u, L.N, P->stream), "zero");
  // ||b|| with a power-of-two prescale taken from max |b|
  int* ex = reinterpret_cast<int*>(P->red_out + 4);
  CK(csff::launch_max_exp(L.b64, L.N, ex, P->stream), "max exponent");
  int eb = 0;
  CK(cudaMemcpyAsync(&eb, ex, sizeof(int), cudaMemcpyDeviceToHost, P->stream), "read exponent");
  CK(cudaStreamSynchronize(P->stream), "sync");
  if (eb >= 4000) {
    csff::set_error("right-hand side is not finite");
    if (in) { std::memset(in, 0, sizeof(*in)); in->status = CSFF_ERR_NONFINITE; }
    return CSFF_ERR_NONFINITE;
  }
  if (eb <= -2000) eb = 0;
  const bool fp64 = P->opts.precision == CSFF_PREC_FP64;
  const bool df = !fp64 && P->opts.refine_fp64 == 0;
  if (!df) {
    CS(norm64(P, L.b64, eb, 1));
  } else {
    // the mixed solve's operands: q (once per coefficient set) and b' = 2^-eb b as
    // double-float pairs, b' rounded to FP32 (the first residual for a zero
    // guess) and ||b'|| from the same pass
    if (!P->dfq_ready) {
      CK(csff::launch_df_split(L.q64, L.N, 0, P->dfq, nullptr, nullptr, nullptr, P->stream), "split q");
      P->dfq_ready = true;
    }
    CK(csff::launch_df_split(L.b64, L.N, -eb, P->dfb, L.b32, P->dfpart, P->red_out + 1, P->stream), "split b");
  }
  CS(read_scalars(P, 2));
  const double nb = df ? std::ldexp(P->red_host[1], eb) : P->red_host[1];
  csff_status st;
  if (nb == 0.0) {
    CK(csff::launch_zero<double>(u, L.N, P->stream), "zero");
    if (in) { std::memset(in, 0, sizeof(*in)); in->n_hist = 1; }
    st = CSFF_OK;
  } else {
    if (fp64) {
      if (use_guess)
        CK(cudaMemcpyAsync(L.u64, u, sizeof(double2) * (size_t)L.N, cudaMemcpyDeviceToDevice, P->stream), "copy");
      else
        CK(csff::launch_zero<double>(L.u64, L.N, P->stream), "zero");
    }
    // the mixed solve reads the guess from u and writes the solution there itself
    st = fp64 ? solve_fp64(P, eb, nb, in) : solve_mixed(P, eb, nb, in, use_guess ? u : nullptr, u);
    if (P->net && !fp64) {
      csff_status nst = csff::net_check(P->net);
      for (int l = 0; l < P->learned_levels && l < 16; ++l)
        if (nst == CSFF_OK && P->level_net[l]) nst = csff::net_check(P->level_net[l]);
      if (nst != CSFF_OK) st = nst;
    }
    if (fp64 && st != CSFF_ERR_CUDA && st != CSFF_ERR_OOM && st != CSFF_ERR_INVALID_ARG)
      CK(cudaMemcpyAsync(u, L.u64, sizeof(double2) * (size_t)L.N, cudaMemcpyDeviceToDevice, P->stream), "copy");
  }
  if (st == CSFF_ERR_CUDA || st == CSFF_ERR_OOM || st == CSFF_ERR_INVALID_ARG) return st;
  if (in) in->status = st;
  return st;
}

csff_status csff_solve_fmg(csff_plan* P, int n_rhs, const double* eta, void* u_dev, int* level_cycles,
                           csff_info* info) {
  if (!P || !eta || !u_dev || n_rhs < 0) return invalid("bad solve arguments");
  if (P->opts.precision != CSFF_PREC_FP64) {
    csff::set_error("full multigrid runs FP64 V-cycles: the plan's precision must be CSFF_PREC_FP64");
    return CSFF_ERR_UNSUPPORTED;
  }
  Level& L = P->lv[0];
  const int nl = (int)P->lv.size();
  int worst = CSFF_OK;
  for (int r = 0; r < n_rhs; ++r) {
    CS(csff_rhs(P, 1, eta + (size_t)r * P->dim, L.b64));
    const csff_status st = fmg_loaded(P, (double2*)u_dev + (size_t)r * L.N,
                                      level_cycles ? level_cycles + (size_t)r * (nl - 1) : nullptr,
                                      info ? info + r : nullptr);
    if (st == CSFF_ERR_CUDA || st == CSFF_ERR_OOM || st == CSFF_ERR_INVALID_ARG) return st;
    worst = worse(worst, st);
  }
  return (csff_status)worst;
}

csff_status csff_solve_rhs(csff_plan* P, const void* b_dev, void* u_dev, int use_guess, csff_info* info) {
  if (!P || !b_dev || !u_dev) return invalid("bad solve arguments");
  Level& L = P->lv[0];
  CK(cudaMemcpyAsync(L.b64, b_dev, sizeof(double2) * (size_t)L.N, cudaMemcpyDeviceToDevice, P->stream), "copy rhs");
  return solve_loaded(P, (double2*)u_dev, use_guess, info);
}

// The coefficients of every level from the finest level's q64 (already set):
// injection to the coarse levels, 1/d and FP32 copies, the coarsest inverse.
static csff_status user_q_levels(csff_plan* P) {
  cudaStream_t s = P->stream;
  for (size_t l = 1; l < P->lv.size(); ++l) CK(csff::launch_inject_q(P->dim, P->lv[l - 1], P->lv[l], s), "inject q");
  for (const Level& L : P->lv) CK(csff::launch_coefs_from_q(P->dim, L, s), "coefficients");
  const Level& Lc = P->lv.back();
  std::vector<double2> qc((size_t)Lc.N);
  CK(cudaMemcpyAsync(qc.data(), Lc.q64, sizeof(double2) * qc.size(), cudaMemcpyDeviceToHost, s), "read q");
  CK(cudaStreamSynchronize(s), "sync");
  std::vector<double2> inv;
  if (!coarse_inverse(P, Lc, inv, &qc)) return invalid("coarsest operator is singular");
  std::vector<float2> inv32(inv.size());
  for (size_t i = 0; i < inv.size(); ++i) inv32[i] = make_float2((float)inv[i].x, (float)inv[i].y);
  CK(cudaMemcpy(P->coarse_inv, inv.data(), sizeof(double2) * inv.size(), cudaMemcpyHostToDevice), "upload inverse");
  CK(cudaMemcpy(P->coarse_inv32, inv32.data(), sizeof(float2) * inv32.size(), cudaMemcpyHostToDevice),
     "upload inverse");
  // the fused FP32 tiles form q from the Gaussian factors: per-level kernels from now on
  P->fused_lc = -1;
  P->user_q = true;
  P->dfq_ready = false;
  destroy_graphs(P);
  return CSFF_OK;
}

csff_status csff_plan_set_potential(csff_plan* P, const void* q_dev) {
  if (!P || !q_dev) return invalid("bad potential arguments");
  CK(cudaMemcpyAsync(P->lv[0].q64, q_dev, sizeof(double2) * (size_t)P->lv[0].N, cudaMemcpyDeviceToDevice,
                     P->stream),
     "copy potential");
  return user_q_levels(P);
}

csff_status csff_plan_set_schroedinger(csff_plan* P, double E, const void* V_dev) {
  if (!P || !V_dev || !std::isfinite(E)) return invalid("bad Schroedinger potential arguments");
  Level& L = P->lv[0];
  CK(csff::launch_affine((const double2*)V_dev, L.N, 2.0 * E, -2.0, L.q64, P->stream), "q = 2E - 2V");
  return user_q_levels(P);
}

csff_status csff_solve_schroedinger(csff_plan* P, const void* phi_dev, void* u_dev, int use_guess, csff_info* info) {
  if (!P || !phi_dev || !u_dev) return invalid("bad solve arguments");
  Level& L = P->lv[0];
  CK(csff::launch_affine((const double2*)phi_dev, L.N, 0.0, 2.0, L.b64, P->stream), "b = 2 phi");
  return solve_loaded(P, (double2*)u_dev, use_guess, info);
}

csff_status csff_far_field(csff_plan* P, int n_rhs, const double* eta, const void* u_dev, int n_ang,
                           const double* alpha, void* F_dev, int32_t* F_exp_dev) {
  if (!P || !eta || !u_dev || !alpha || !F_dev || n_rhs < 0 || n_ang < 0) return invalid("bad far-field arguments");
  if (n_ang == 0 || n_rhs == 0) return CSFF_OK;
  Level& L = P->lv[0];
  bool any_scaled = false;
  for (int r = 0; r < n_rhs; ++r) {
    bool scaled = false;
    CS(csff::far_field_one(P, eta + (size_t)r * P->dim, (const double2*)u_dev + (size_t)r * L.N, n_ang, alpha,
                           (double2*)F_dev + (size_t)r * n_ang, F_exp_dev ? F_exp_dev + (size_t)r * n_ang : nullptr,
                           F_exp_dev ? nullptr : &scaled));
    any_scaled |= scaled;
  }
  return any_scaled ? CSFF_WARN_ILL_CONDITIONED : CSFF_OK;
}

csff_status csff_far_field_work(csff_plan* P, double* executed) {
  if (!P || !executed) return invalid("bad far-field work arguments");
  return csff::far_field_executed(P, executed);
}

csff_status csff_plan_set_far_field_mode(csff_plan* P, int mode) {
  if (!P || (mode != CSFF_FF_FP64 && mode != CSFF_FF_TC_BF16X4)) return invalid("bad far-field mode");
  P->ff_mode = mode;
  return CSFF_OK;
}

csff_status csff_residual(csff_plan* P, int level, int arith, const void* u, const void* b, void* r) {
  CS(check_level(P, level, arith));
  if (!u || !b || !r) return invalid("NULL buffer");
  Level& L = P->lv[level];
  if (arith == CSFF_ARITH_FP64)
    CK(csff::launch_residual<double>(P->dim, L, (const double2*)u, (const double2*)b, (double2*)r, P->stream), "residual");
  else
    CK(csff::launch_residual<float>(P->dim, L, (const float2*)u, (const float2*)b, (float2*)r, P->stream), "residual");
  return CSFF_OK;
}

csff_status csff_smooth(csff_plan* P, int level, int arith, void* u, const void* b, int sweeps) {
  CS(check_level(P, level, arith));
  if (!u || !b || sweeps < 0) return invalid("bad smoother arguments");
  if (arith == CSFF_ARITH_FP64) return smooth<double>(P, level, (double2*)u, (const double2*)b, sweeps);
  return smooth<float>(P, level, (float2*)u, (const float2*)b, sweeps);
}

csff_status csff_restrict(csff_plan* P, int level, int arith, const void* rf, void* bc) {
  CS(check_level(P, level, arith));
  if (level + 1 >= (int)P->lv.size()) return invalid("no coarser level");
  if (!rf || !bc) return invalid("NULL buffer");
  Level& F = P->lv[level];
  Level& C = P->lv[level + 1];
  if (arith == CSFF_ARITH_FP64)
    CK(csff::launch_restrict<double>(P->dim, F, C, (const double2*)rf, (double2*)bc, P->stream), "restrict");
  else
    CK(csff::launch_restrict<float>(P->dim, F, C, (const float2*)rf, (float2*)bc, P->stream), "restrict");
  return CSFF_OK;
}

csff_status csff_prolong_add(csff_plan* P, int level, int arith, const void* ec, void* uf) {
  CS(check_level(P, level, arith));
  if (level + 1 >= (int)P->lv.size()) return invalid("no coarser level");
  if (!ec || !uf) return invalid("NULL buffer");
  Level& F = P->lv[level];
  Level& C = P->lv[level + 1];
  if (arith == CSFF_ARITH_FP64)
    CK(csff::launch_prolong_add<double>(P->dim, F, C, (const double2*)ec, (double2*)uf, P->stream), "prolong");
  else
    CK(csff::launch_prolong_add<float>(P->dim, F, C, (const float2*)ec, (float2*)uf, P->stream), "prolong");
  return CSFF_OK;
}

csff_status csff_coarse_solve(csff_plan* P, int arith, const void* b, void* u) {
  CS(check_level(P, 0, arith));
  if (!b || !u) return invalid("NULL buffer");
  if (arith == CSFF_ARITH_FP64)
    CK(csff::launch_coarse_solve<double>(P->coarse_inv, P->coarse_N, (const double2*)b, (double2*)u, P->stream),
       "coarse");
  else
    CK(csff::launch_coarse_solve<float>(P->coarse_inv32, P->coarse_N, (const float2*)b, (float2*)u, P->stream),
       "coarse");
  return CSFF_OK;
}

csff_status csff_norm2(csff_plan* P, int level, int arith, const void* v, double* out) {
  CS(check_level(P, level, arith));
  if (!v || !out) return invalid("NULL argument");
  Level& L = P->lv[level];
  if (arith == CSFF_ARITH_FP64)
    CK(csff::launch_norm2<double>((const double2*)v, L.N, 0, P->red, P->red_blocks, P->red_out + 2, P->stream),
       "norm");
  else
    CK(csff::launch_norm2<float>((const float2*)v, L.N, 0, P->red, P->red_blocks, P->red_out + 2, P->stream),
       "norm");
  CS(read_scalars(P, 3));
  *out = P->red_host[2];
  return CSFF_OK;
}

csff_status csff_vcycle(csff_plan* P, int arith, void* u, const void* b) {
  CS(check_level(P, 0, arith));
  if (!u || !b) return invalid("NULL buffer");
  if (arith == CSFF_ARITH_FP64) return run_vcycle<double>(P, (double2*)u, (const double2*)b, false);
  return run_vcycle<float>(P, (float2*)u, (const float2*)b, false);
}

}  // extern "C"
