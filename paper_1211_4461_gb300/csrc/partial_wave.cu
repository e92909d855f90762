// Partial-wave Schroedinger problem on the complex contour (Sec. 5.2-5.3):
// the one-dimensional functions of eqs. (boundstate) and (testfunction)
// along the rotated axis, and the separable contour integrals of eqs.
// (single-ionization) and (double-ionization).
//
// The 1D functions are plan-time work of O(m) per function on the host: a
// complex tridiagonal solve per inverse-iteration step for a bound state, one
// three-term recurrence for a regular solution.  The integrals run on the
// device: out[r] = e^{2 i gamma} h^2 sum_{j,i} X[r][i] Y[r][j] g[j][i] with
// g = f - w u formed on the fly, as a complex FP64 product T = X g^T (shared-
// memory tiles) followed by one row dot product out[r] = s sum_j Y[r][j] T[r][j].
#include <cmath>
#include <complex>
#include <vector>

#include "csff_internal.h"

namespace csff {
namespace {

using cd = std::complex<double>;

// ---- device: separable contour integrals --------------------------------------
constexpr int ST = 16;   // tile edge of the product T = X g^T

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// T[r][j] = sum_i X[r][i] g[j][i], g = f - w u (w, u may be null: g = f)
__global__ void k_sep_product(const double2* __restrict__ X, int R, const double2* __restrict__ f,
                              const double2* __restrict__ w, const double2* __restrict__ u, int m,
                              double2* __restrict__ T) {
  __shared__ double2 Xs[ST][ST + 1];
  __shared__ double2 Gs[ST][ST + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = blockIdx.y * ST + ty, j = blockIdx.x * ST + tx;
  double2 acc = make_double2(0.0, 0.0);
  for (int i0 = 0; i0 < m; i0 += ST) {
    const int xi = i0 + tx;
    Xs[ty][tx] = (r < R && xi < m) ? X[(long long)r * m + xi] : make_double2(0.0, 0.0);
    const int gj = blockIdx.x * ST + ty, gi = i0 + tx;   // row gj of g, column gi
    double2 g = make_double2(0.0, 0.0);
    if (gj < m && gi < m) {
      const long long o = (long long)gj * m + gi;
      g = f[o];
      if (w && u) {
        const double2 p = zmul(w[o], u[o]);
        g = make_double2(g.x - p.x, g.y - p.y);
      }
    }
    Gs[ty][tx] = g;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < ST; ++t) {
      const double2 p = zmul(Xs[ty][t], Gs[tx][t]);
      acc.x += p.x;
      acc.y += p.y;
    }
    __syncthreads();
  }
  if (r < R && j < m) T[(long long)r * m + j] = acc;
}

// out[r] = s * sum_j Y[r][j] T[r][j]: one block per row
__global__ void k_sep_rows(const double2* __restrict__ Y, const double2* __restrict__ T, int m, double2 s,
                           double2* __restrict__ out) {
  __shared__ double shr[32], shi[32];
  const int r = blockIdx.x;
  double ar = 0.0, ai = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double2 p = zmul(Y[(long long)r * m + j], T[(long long)r * m + j]);
    ar += p.x;
    ai += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
  }
  const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { shr[wid] = ar; shi[wid] = ai; }
  __syncthreads();
  if (wid == 0) {
    ar = (l < (int)(blockDim.x >> 5)) ? shr[l] : 0.0;
    ai = (l < (int)(blockDim.x >> 5)) ? shi[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (l == 0) out[r] = zmul(s, make_double2(ar, ai));
  }
}

// ---- host: 1D functions along the contour ---------------------------------------
// H1 = -1/2 d^2/dz^2 + V on z_i = i h_z (i = 1..m, Dirichlet at 0 and m+1):
// diagonal 1/h_z^2 + V_i, off-diagonal -1/(2 h_z^2).  Solves (H1 - s) y = x by
// elimination down the tridiagonal system (returns false on a zero pivot).
bool tri_solve(const std::vector<cd>& dg, cd off, cd s, const std::vector<cd>& x, std::vector<cd>& y) {
  const int m = (int)dg.size();
  std::vector<cd> c(m), d(m);
  cd piv = dg[0] - s;
  if (piv == 0.0) return false;
  c[0] = off / piv;
  d[0] = x[0] / piv;
  for (int i = 1; i < m; ++i) {
    piv = dg[i] - s - off * c[i - 1];
    if (piv == 0.0) return false;
    c[i] = off / piv;
    d[i] = (x[i] - off * d[i - 1]) / piv;
  }
  y.assign(m, cd(0, 0));
  y[m - 1] = d[m - 1];
  for (int i = m - 2; i >= 0; --i) y[i] = d[i] - c[i] * y[i + 1];
  return true;
}

cd bilinear_rq(const std::vector<cd>& dg, cd off, const std::vector<cd>& y) {
  const int m = (int)y.size();
  cd num(0, 0), den(0, 0);
  for (int i = 0; i < m; ++i) {
    cd hy = dg[i] * y[i];
    if (i > 0) hy += off * y[i - 1];
    if (i + 1 < m) hy += off * y[i + 1];
    num += y[i] * hy;
    den += y[i] * y[i];
  }
  return num / den;
}

}  // namespace

// Sec. 5.2: (-1/2 Delta + V - E) u = phi times 2 is the plan's A u = c (2d u -
// sum_nbr u) - q u = b with q = 2E - 2V and b = 2 phi; out = a + s v per point
// (a = 2E, s = -2 for q; a = 0, s = 2 for b).  Both scalings are exact.
__global__ void k_affine(const double2* __restrict__ v, long long N, double a, double s, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double2 x = v[i];
    out[i] = make_double2(fma(s, x.x, a), s * x.y);
  }
}

cudaError_t launch_affine(const double2* v, long long N, double a, double s, double2* out, cudaStream_t st) {
  const int blk = 256;
  const long long want = (N + blk - 1) / blk;
  const int grid = (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
  k_affine<<<grid, blk, 0, st>>>(v, N, a, s, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace csff

using csff::cd;

extern "C" {

csff_status csff_contour_bound_state(int m, double h, double gamma, const double* v, double lambda_guess,
                                     double* lambda, double* phi) {
  if (m < 3 || !(h > 0.0) || !v || !lambda || !phi) {
    csff::set_error("bad bound-state arguments");
    return CSFF_ERR_INVALID_ARG;
  }
  const cd hz = h * std::polar(1.0, gamma);
  const cd off = -0.5 / (hz * hz);
  std::vector<cd> dg(m);
  for (int i = 0; i < m; ++i) dg[i] = 1.0 / (hz * hz) + cd(v[2 * i], v[2 * i + 1]);
  std::vector<cd> x(m, cd(1.0, 0.0)), y;
  cd s(lambda_guess, 0.0);
  // a few steps with the fixed shift, then Rayleigh-quotient updates
  bool done = false;
  for (int it = 0; it < 200 && !done; ++it) {
    if (!csff::tri_solve(dg, off, s, x, y)) {
      s += cd(1e-12 * (1.0 + std::abs(s)), 0.0);
      continue;
    }
    double mx = 0.0;
    for (const cd& a : y) mx = std::max(mx, std::abs(a));
    if (!(mx > 0.0) || !std::isfinite(mx)) break;
    for (int i = 0; i < m; ++i) x[i] = y[i] / mx;
    const cd rq = csff::bilinear_rq(dg, off, x);
    if (it >= 4) {
      done = std::abs(rq - s) <= 1e-14 * std::max(1.0, std::abs(rq));
      s = rq;
    }
  }
  if (!done) {
    csff::set_error("bound-state iteration did not converge");
    return CSFF_ERR_NOT_CONVERGED;
  }
  // normalise: sum_i phi_i^2 h_z = 1 (no conjugate), largest entry real-positive
  cd nrm(0, 0);
  for (const cd& a : x) nrm += a * a;
  nrm = std::sqrt(nrm * hz);
  int jmax = 0;
  for (int i = 0; i < m; ++i) {
    x[i] /= nrm;
    if (std::abs(x[i]) > std::abs(x[jmax])) jmax = i;
  }
  const double sg = x[jmax].real() < 0.0 ? -1.0 : 1.0;
  for (int i = 0; i < m; ++i) {
    phi[2 * i] = sg * x[i].real();
    phi[2 * i + 1] = sg * x[i].imag();
  }
  lambda[0] = s.real();
  lambda[1] = s.imag();
  return CSFF_OK;
}

csff_status csff_contour_regular_solution(int m, double h, double gamma, const double* v, double k, double tail,
                                          double* phi) {
  if (m < 3 || !(h > 0.0) || !(k > 0.0) || !(tail > 0.0) || !v || !phi) {
    csff::set_error("bad regular-solution arguments");
    return CSFF_ERR_INVALID_ARG;
  }
  const cd hz = h * std::polar(1.0, gamma);
  // p_0 = 0, p_1 = h_z, p_{i+1} = 2 p_i - p_{i-1} + 2 h_z^2 (V_i - k^2/2) p_i
  std::vector<cd> p(m + 1, cd(0, 0));
  p[1] = hz;
  for (int i = 1; i < m; ++i) {
    const cd vi(v[2 * (i - 1)], v[2 * (i - 1) + 1]);
    p[i + 1] = 2.0 * p[i] - p[i - 1] + 2.0 * hz * hz * (vi - 0.5 * k * k) * p[i];
  }
  int i0 = -1;
  for (int i = 1; i < m; ++i)
    if (std::abs(cd(v[2 * (i - 1)], v[2 * (i - 1) + 1])) < tail) { i0 = i; break; }
  if (i0 < 0) {
    csff::set_error("the potential does not fall below the tail threshold inside the contour");
    return CSFF_ERR_INVALID_ARG;
  }
  // where V has died out, p_i = a e^{i theta i} + b e^{-i theta i} with
  // cos theta = 1 - (k h_z)^2 / 2 (Im theta >= 0); p = 2 sqrt(ab) sin(theta i + delta)
  cd th = std::acos(1.0 - 0.5 * (k * hz) * (k * hz));
  if (th.imag() < 0.0) th = -th;
  const cd I(0, 1);
  const cd e00 = std::exp(I * th * (double)i0), e01 = std::exp(-I * th * (double)i0);
  const cd e10 = std::exp(I * th * (double)(i0 + 1)), e11 = std::exp(-I * th * (double)(i0 + 1));
  const cd det = e00 * e11 - e01 * e10;
  const cd a = (p[i0] * e11 - e01 * p[i0 + 1]) / det;
  const cd b = (e00 * p[i0 + 1] - e10 * p[i0]) / det;
  const cd amp = 2.0 * std::sqrt(a * b) * std::sqrt(k);
  for (int i = 0; i < m; ++i) {
    const cd q = p[i + 1] / amp;
    phi[2 * i] = q.real();
    phi[2 * i + 1] = q.imag();
  }
  return CSFF_OK;
}

csff_status csff_separable_sum(csff_plan* P, int n_rows, const void* X, const void* Y, const void* f,
                               const void* w, const void* u, void* out) {
  if (!P || n_rows < 0 || !X || !Y || !f || !out || (!w) != (!u)) {
    csff::set_error("bad separable-sum arguments");
    return CSFF_ERR_INVALID_ARG;
  }
  if (P->dim != 2) {
    csff::set_error("separable sums are two-dimensional");
    return CSFF_ERR_INVALID_ARG;
  }
  if (n_rows == 0) return CSFF_OK;
  const csff::Level& L = P->lv[0];
  const int m = L.m;
  const size_t need = (size_t)n_rows * m;
  if (need > P->sep_cap) {
    if (P->sep_T) cudaFree(P->sep_T);
    P->sep_T = nullptr;
    P->sep_cap = 0;
    cudaError_t e = cudaMalloc((void**)&P->sep_T, sizeof(double2) * need);
    if (e != cudaSuccess) return csff::cuda_fail(e, "separable-sum scratch");
    P->sep_cap = need;
  }
  const cd sc = std::polar(L.h * L.h, 2.0 * P->prob.gamma);
  dim3 g((m + csff::ST - 1) / csff::ST, (n_rows + csff::ST - 1) / csff::ST), b(csff::ST, csff::ST);
  csff::k_sep_product<<<g, b, 0, P->stream>>>((const double2*)X, n_rows, (const double2*)f, (const double2*)w,
                                               (const double2*)u, m, P->sep_T);
  csff::k_sep_rows<<<n_rows, 256, 0, P->stream>>>((const double2*)Y, P->sep_T, m,
                                                  make_double2(sc.real(), sc.imag()), (double2*)out);
  csff::count_launch(2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CSFF_OK : csff::cuda_fail(e, "separable sum");
}

}  // extern "C"
