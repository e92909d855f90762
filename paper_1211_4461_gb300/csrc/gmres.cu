// GMRES(m) cycles as the multigrid smoother (Sec. 3.3: a Krylov method such
// as GMRES(m), m = 2 or 3, replaces omega-Jacobi / Gauss-Seidel smoothing so
// that rotation angles near 10 degrees stay stable; Tables 2-3 use GMRES(3)
// at gamma = 9.9 degrees).  One smoothing step from the iterate u:
//
//   r0 = b - A u,  beta = ||r0||,  v_0 = r0 / beta
//   for j < m:  w = A v_j;  for i <= j: h_ij = (v_i, w), w -= h_ij v_i
//               (modified Gram-Schmidt);  h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j}
//   y = argmin_y || beta e_1 - H y ||_2  (complex Givens rotations),  u += V y
//
// w is formed in the slot of v_{j+1}, so the m+1 basis vectors are the only
// level-sized scratch.  Every step is a kernel on the plan's stream: inner
// products reduce per block into partial sums and one block sums those into
// the Hessenberg matrix in device memory, and one thread solves the small
// least-squares problem, so a smoothing step is graph-capturable and never
// synchronises with the host.  Inner products and norms accumulate in FP64
// for both cycle precisions.  A zero h_{j+1,j} (the Krylov space is
// invariant: the Arnoldi process breaks down) leaves v_{j+1} = 0 and the
// least-squares step uses the first j+1 columns only.
#include "csff_internal.h"

namespace csff {
namespace {

constexpr int GT = 256;            // threads of the 1D kernels
constexpr int BX = 32, BY = 8;     // apply kernel block (x, y); blockIdx.z = z plane

__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }

// sum over the block; valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// w = A v with (A v)_j = c (2d v_j - sum_nbr v) - q_j v_j (neighbours outside
// the interior are zero)
template <typename T, int D>
__global__ void k_gm_apply(const cx<T>* __restrict__ v, const cx<T>* __restrict__ q, cx<T> c, int m,
                           cx<T>* __restrict__ w) {
  pdl_prologue();
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  const int iz = (D == 3) ? (int)blockIdx.z : 0;
  if (ix >= m || iy >= m) return;
  const long long idx = ((long long)iz * m + iy) * m + ix;
  using C = cx<T>;
  C s = mk<C>(0, 0);
  if (ix > 0) s = cadd(s, v[idx - 1]);
  if (ix < m - 1) s = cadd(s, v[idx + 1]);
  if (iy > 0) s = cadd(s, v[idx - m]);
  if (iy < m - 1) s = cadd(s, v[idx + m]);
  if (D == 3) {
    const long long p = (long long)m * m;
    if (iz > 0) s = cadd(s, v[idx - p]);
    if (iz < m - 1) s = cadd(s, v[idx + p]);
  }
  const C vj = v[idx];
  w[idx] = csub(cmul(c, csub(cscale(vj, (T)(2 * D)), s)), cmul(q[idx], vj));
}

// per-block partial sums of (x, y) = sum conj(x_i) y_i
template <typename T>
__global__ void k_gm_dot_partial(const cx<T>* __restrict__ x, const cx<T>* __restrict__ y, long long N,
                                 double2* __restrict__ part) {
  pdl_prologue();
  __shared__ double sh[32];
  double ar = 0.0, ai = 0.0;
  for (long long i = blockIdx.x * (long long)GT + threadIdx.x; i < N; i += (long long)gridDim.x * GT) {
    const double xr = x[i].x, xi = x[i].y, yr = y[i].x, yi = y[i].y;
    ar = fma(xr, yr, fma(xi, yi, ar));
    ai = fma(xr, yi, fma(-xi, yr, ai));
  }
  ar = block_sum(ar, sh);
  ai = block_sum(ai, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(ar, ai);
}

// H[i][j] = sum of the partials
__global__ void k_gm_dot_finish(const double2* __restrict__ part, int nb, GmState* __restrict__ S, int i, int j) {
  pdl_prologue();
  __shared__ double sh[32];
  double ar = 0.0, ai = 0.0;
  for (int t = threadIdx.x; t < nb; t += GT) {
    ar += part[t].x;
    ai += part[t].y;
  }
  ar = block_sum(ar, sh);
  ai = block_sum(ai, sh);
  if (threadIdx.x == 0) S->H[i][j] = make_double2(ar, ai);
}

// nrm[slot] = sqrt(sum of the partials' real parts), inv[slot] = 1 / nrm (0 for
// a zero norm); for slot > 0 also H[slot][slot-1] = nrm
__global__ void k_gm_norm_finish(const double2* __restrict__ part, int nb, GmState* __restrict__ S, int slot) {
  pdl_prologue();
  __shared__ double sh[32];
  double a = 0.0;
  for (int t = threadIdx.x; t < nb; t += GT) a += part[t].x;
  a = block_sum(a, sh);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(a);
    S->nrm[slot] = nrm;
    S->inv[slot] = nrm > 0.0 ? 1.0 / nrm : 0.0;
    if (slot > 0) S->H[slot][slot - 1] = make_double2(nrm, 0.0);
  }
}

// v *= inv[slot]
template <typename T>
__global__ void k_gm_scale(cx<T>* __restrict__ v, long long N, const GmState* __restrict__ S, int slot) {
  pdl_prologue();
  const double s = S->inv[slot];
  for (long long i = blockIdx.x * (long long)GT + threadIdx.x; i < N; i += (long long)gridDim.x * GT)
    v[i] = mk<cx<T>>((T)(v[i].x * s), (T)(v[i].y * s));
}

// w -= H[i][j] v
template <typename T>
__global__ void k_gm_axpy(cx<T>* __restrict__ w, const cx<T>* __restrict__ v, long long N,
                          const GmState* __restrict__ S, int i, int j) {
  pdl_prologue();
  const double2 h = S->H[i][j];
  for (long long t = blockIdx.x * (long long)GT + threadIdx.x; t < N; t += (long long)gridDim.x * GT) {
    const double vr = v[t].x, vi = v[t].y;
    w[t] = mk<cx<T>>((T)(w[t].x - (h.x * vr - h.y * vi)), (T)(w[t].y - (h.x * vi + h.y * vr)));
  }
}

// y = argmin || beta e_1 - H y ||_2 over the first k columns (k = m, or the
// column after which the Arnoldi process broke down), by complex Givens
// rotations G_j = [c s; -conj(s) c] with c = |a|/r, s = (a/|a|) conj(b)/r,
// r = sqrt(|a|^2 + |b|^2), which zero the subdiagonal entry b under a, then
// back substitution.  One thread.
__global__ void k_gm_lsq(GmState* __restrict__ S, int m) {
  pdl_prologue();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = m;
  if (!(S->nrm[0] > 0.0)) k = 0;
  for (int j = 0; j < k; ++j)
    if (S->nrm[j + 1] == 0.0) {
      k = j + 1;
      break;
    }
  double2 R[GM_MAX + 1][GM_MAX], g[GM_MAX + 1];
  for (int i = 0; i <= m; ++i) {
    for (int j = 0; j < m; ++j) R[i][j] = S->H[i][j];
    g[i] = make_double2(i == 0 ? S->nrm[0] : 0.0, 0.0);
  }
  for (int j = 0; j < k; ++j) {
    const double2 a = R[j][j], b = R[j + 1][j];
    const double na = hypot(a.x, a.y), nb = hypot(b.x, b.y), r = hypot(na, nb);
    double c;
    double2 s;
    if (r == 0.0) {
      c = 1.0;
      s = make_double2(0.0, 0.0);
    } else if (na == 0.0) {
      c = 0.0;
      s = make_double2(1.0, 0.0);
    } else {
      c = na / r;
      const double2 ph = make_double2(a.x / na, a.y / na);
      const double2 t = dmul(ph, dconj(b));
      s = make_double2(t.x / r, t.y / r);
    }
    const double2 sc = dconj(s);
    for (int col = j; col < k; ++col) {
      const double2 x = R[j][col], z = R[j + 1][col];
      const double2 sz = dmul(s, z), scx = dmul(sc, x);
      R[j][col] = make_double2(c * x.x + sz.x, c * x.y + sz.y);
      R[j + 1][col] = make_double2(c * z.x - scx.x, c * z.y - scx.y);
    }
    const double2 gx = g[j], gz = g[j + 1];
    const double2 sgz = dmul(s, gz), scgx = dmul(sc, gx);
    g[j] = make_double2(c * gx.x + sgz.x, c * gx.y + sgz.y);
    g[j + 1] = make_double2(c * gz.x - scgx.x, c * gz.y - scgx.y);
  }
  double2 y[GM_MAX];
  for (int j = GM_MAX - 1; j >= 0; --j) y[j] = make_double2(0.0, 0.0);
  for (int j = k - 1; j >= 0; --j) {
    double2 t = g[j];
    for (int col = j + 1; col < k; ++col) {
      const double2 p = dmul(R[j][col], y[col]);
      t = make_double2(t.x - p.x, t.y - p.y);
    }
    const double2 d = R[j][j];
    const double dd = d.x * d.x + d.y * d.y;
    y[j] = dd > 0.0 ? make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd)
                    : make_double2(0.0, 0.0);
  }
  for (int j = 0; j < GM_MAX; ++j) S->y[j] = y[j];
  S->k = k;
}

// u += sum_{j < k} y_j v_j
template <typename T>
__global__ void k_gm_update(cx<T>* __restrict__ u, const cx<T>* __restrict__ V, long long N,
                            const GmState* __restrict__ S) {
  pdl_prologue();
  const int k = S->k;
  double2 y[GM_MAX];
  for (int j = 0; j < GM_MAX; ++j) y[j] = S->y[j];
  for (long long i = blockIdx.x * (long long)GT + threadIdx.x; i < N; i += (long long)gridDim.x * GT) {
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < k; ++j) {
      const cx<T> v = V[(long long)j * N + i];
      ar += y[j].x * (double)v.x - y[j].y * (double)v.y;
      ai += y[j].x * (double)v.y + y[j].y * (double)v.x;
    }
    u[i] = mk<cx<T>>((T)((double)u[i].x + ar), (T)((double)u[i].y + ai));
  }
}

template <typename T> const cx<T>* qtab_of(const Level& L);
template <> const double2* qtab_of<double>(const Level& L) { return L.q64; }
template <> const float2* qtab_of<float>(const Level& L) { return L.q32; }

int blocks_for(long long N, int cap) {
  const long long need = (N + GT - 1) / GT;
  return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

}  // namespace

template <typename T>
cudaError_t launch_gmres_step(int dim, const Level& L, int m, cx<T>* u, const cx<T>* b, cx<T>* V,
                              double2* part, int part_cap, GmState* S, cudaStream_t s) {
  if (m < 1 || m > GM_MAX) return cudaErrorInvalidValue;
  const long long N = L.N;
  const int nb = blocks_for(N, part_cap);
  const cx<T> c = mk<cx<T>>((T)L.c.x, (T)L.c.y);
  const dim3 ga((L.m + BX - 1) / BX, (L.m + BY - 1) / BY, dim == 3 ? L.m : 1), ba(BX, BY);
  ProfScope ps(mg_family<T>(), s, 0, 0);
  cudaError_t e = cudaSuccess;
  int launches = 0;
  auto ok = [&](cudaError_t r) {
    ++launches;
    if (e == cudaSuccess) e = r;
  };
  auto norm_into = [&](const cx<T>* x, int slot) {
    ok(launch_pdl(k_gm_dot_partial<T>, dim3(nb), dim3(GT), 0, s, x, x, N, part));
    ok(launch_pdl(k_gm_norm_finish, dim3(1), dim3(GT), 0, s, (const double2*)part, nb, S, slot));
  };
  // r0 = b - A u, beta, v_0
  if ((e = launch_residual<T>(dim, L, u, b, V, s)) != cudaSuccess) return e;
  norm_into(V, 0);
  ok(launch_pdl(k_gm_scale<T>, dim3(nb), dim3(GT), 0, s, V, N, (const GmState*)S, 0));
  for (int j = 0; j < m; ++j) {
    const cx<T>* vj = V + (long long)j * N;
    cx<T>* w = V + (long long)(j + 1) * N;
    if (dim == 2) ok(launch_pdl(k_gm_apply<T, 2>, ga, ba, 0, s, vj, qtab_of<T>(L), c, L.m, w));
    else ok(launch_pdl(k_gm_apply<T, 3>, ga, ba, 0, s, vj, qtab_of<T>(L), c, L.m, w));
    for (int i = 0; i <= j; ++i) {
      const cx<T>* vi = V + (long long)i * N;
      ok(launch_pdl(k_gm_dot_partial<T>, dim3(nb), dim3(GT), 0, s, vi, (const cx<T>*)w, N, part));
      ok(launch_pdl(k_gm_dot_finish, dim3(1), dim3(GT), 0, s, (const double2*)part, nb, S, i, j));
      ok(launch_pdl(k_gm_axpy<T>, dim3(nb), dim3(GT), 0, s, w, vi, N, (const GmState*)S, i, j));
    }
    norm_into(w, j + 1);
    if (j + 1 < m) ok(launch_pdl(k_gm_scale<T>, dim3(nb), dim3(GT), 0, s, w, N, (const GmState*)S, j + 1));
  }
  ok(launch_pdl(k_gm_lsq, dim3(1), dim3(32), 0, s, S, m));
  ok(launch_pdl(k_gm_update<T>, dim3(nb), dim3(GT), 0, s, u, (const cx<T>*)V, N, (const GmState*)S));
  count_launch(launches);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template cudaError_t launch_gmres_step<double>(int, const Level&, int, double2*, const double2*, double2*, double2*,
                                               int, GmState*, cudaStream_t);
template cudaError_t launch_gmres_step<float>(int, const Level&, int, float2*, const float2*, float2*, double2*, int,
                                              GmState*, cudaStream_t);

}  // namespace csff
