// Multigrid kernels on the rotated grid (Sec. 3.2 eq. (csg) with the Sec. 5.2
// stencil; Sec. 4 V-cycle components).  Templated on the real type (double for
// the plain and refinement path, float for the inner cycles of the mixed
// path) and on the dimension.
//
// Layout: m^d interior unknowns, x fastest, interleaved complex.  Boundary
// nodes are not stored (homogeneous Dirichlet).  Grid mapping: block (32, 8)
// over (x, y), blockIdx.z = z plane in 3D.
#include "csff_internal.h"
#include "df_bits.cuh"

namespace csff {
namespace {

constexpr int BX = 32, BY = 8;

template <int D>
__device__ __forceinline__ bool thread_point(int m, int& ix, int& iy, int& iz, long long& idx) {
  ix = blockIdx.x * BX + threadIdx.x;
  iy = blockIdx.y * BY + threadIdx.y;
  iz = (D == 3) ? (int)blockIdx.z : 0;
  if (ix >= m || iy >= m) return false;
  idx = ((long long)iz * m + iy) * m + ix;
  return true;
}

// (A u)_j = c (2d u_j - sum_nbr u) - q_j u_j ; neighbours outside the
// interior are zero.
template <typename T, int D>
__device__ __forceinline__ cx<T> apply_point(const cx<T>* __restrict__ u, cx<T> uj, cx<T> qj, cx<T> c,
                                             int m, int ix, int iy, int iz, long long idx) {
  using C = cx<T>;
  C s = mk<C>(0, 0);
  if (ix > 0) s = cadd(s, u[idx - 1]);
  if (ix < m - 1) s = cadd(s, u[idx + 1]);
  if (iy > 0) s = cadd(s, u[idx - m]);
  if (iy < m - 1) s = cadd(s, u[idx + m]);
  if (D == 3) {
    long long p = (long long)m * m;
    if (iz > 0) s = cadd(s, u[idx - p]);
    if (iz < m - 1) s = cadd(s, u[idx + p]);
  }
  C t = csub(cscale(uj, (T)(2 * D)), s);
  return csub(cmul(c, t), cmul(qj, uj));
}

template <typename T, int D>
__global__ void k_residual(const cx<T>* __restrict__ u, const cx<T>* __restrict__ b,
                           const cx<T>* __restrict__ q, cx<T> c, int m, cx<T>* __restrict__ r) {
  pdl_prologue();
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(m, ix, iy, iz, idx)) return;
  cx<T> au = apply_point<T, D>(u, u[idx], q[idx], c, m, ix, iy, iz, idx);
  r[idx] = csub(b[idx], au);
}

template <typename T, int D>
__global__ void k_jacobi(const cx<T>* __restrict__ u, const cx<T>* __restrict__ b,
                         const cx<T>* __restrict__ q, const cx<T>* __restrict__ dinv, cx<T> c, T omega,
                         int m, cx<T>* __restrict__ u_out) {
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(m, ix, iy, iz, idx)) return;
  cx<T> uj = u[idx];
  cx<T> rj = csub(b[idx], apply_point<T, D>(u, uj, q[idx], c, m, ix, iy, iz, idx));
  u_out[idx] = cadd(uj, cscale(cmul(dinv[idx], rj), omega));
}

// One colour of red-black Gauss-Seidel, in place.  colour 0 (red) = even sum
// of node indices (interior index + 1 per axis).  One thread per point of the
// colour: x thread t of a row takes ix = 2 t + (colour + iy + iz + D) mod 2.
// With d = 2 D c - q the point's equation (A u)_j = d u_j - c sum_nbr u = b_j
// solved for u_j: u_j <- d^{-1} (b_j + c sum_nbr u), which reads neither q nor
// the point's old value.
template <typename T, int D>
__global__ void k_rbgs(cx<T>* u, const cx<T>* __restrict__ b, const cx<T>* __restrict__ dinv, cx<T> c, int m,
                       int colour) {
  const int iy = blockIdx.y * BY + threadIdx.y;
  const int iz = (D == 3) ? (int)blockIdx.z : 0;
  const int ix = 2 * (int)(blockIdx.x * BX + threadIdx.x) + ((colour + iy + iz + D) & 1);
  if (ix >= m || iy >= m) return;
  const long long idx = ((long long)iz * m + iy) * m + ix;
  using C = cx<T>;
  C s = mk<C>(0, 0);
  if (ix > 0) s = cadd(s, u[idx - 1]);
  if (ix < m - 1) s = cadd(s, u[idx + 1]);
  if (iy > 0) s = cadd(s, u[idx - m]);
  if (iy < m - 1) s = cadd(s, u[idx + m]);
  if (D == 3) {
    const long long p = (long long)m * m;
    if (iz > 0) s = cadd(s, u[idx - p]);
    if (iz < m - 1) s = cadd(s, u[idx + p]);
  }
  u[idx] = cmul(dinv[idx], cadd(b[idx], cmul(c, s)));
}

// Full weighting: coarse interior P <- sum over offsets o in {-1,0,1}^d of
// prod(1/2 if o = 0 else 1/4) * r_f[2P + 1 + o].
template <typename T, int D>
__global__ void k_restrict(const cx<T>* __restrict__ rf, int mf, cx<T>* __restrict__ bc, int mc) {
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(mc, ix, iy, iz, idx)) return;
  using C = cx<T>;
  C acc = mk<C>(0, 0);
  const int fx = 2 * ix + 1, fy = 2 * iy + 1, fz = (D == 3) ? 2 * iz + 1 : 0;
  const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
#pragma unroll
  for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz) {
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
      C row = mk<C>(0, 0);
      long long base = ((long long)(fz + oz) * mf + (fy + oy)) * mf + fx;
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) row = cadd(row, cscale(rf[base + ox], w1[ox + 1]));
      T wz = (D == 3) ? w1[oz + 1] : (T)1;
      acc = cadd(acc, cscale(row, w1[oy + 1] * wz));
    }
  }
  bc[idx] = acc;
}

// Linear interpolation weights of fine interior index p along one axis: node
// i = p + 1; even i sits on coarse node i/2 (weight 1), odd i between coarse
// nodes (i-1)/2 and (i+1)/2 (weights 1/2).  Returns the number of coarse
// interior neighbours (coarse interior index = coarse node - 1).
template <typename T>
__device__ __forceinline__ int interp_1d(int p, int mc, int* ci, T* w) {
  int i = p + 1, n = 0;
  if ((i & 1) == 0) {
    int I = i >> 1;
    if (I >= 1 && I <= mc) { ci[n] = I - 1; w[n] = (T)1; ++n; }
  } else {
    int I0 = (i - 1) >> 1, I1 = I0 + 1;
    if (I0 >= 1 && I0 <= mc) { ci[n] = I0 - 1; w[n] = (T)0.5; ++n; }
    if (I1 >= 1 && I1 <= mc) { ci[n] = I1 - 1; w[n] = (T)0.5; ++n; }
  }
  return n;
}

// u_f += P e by coarse cells: cell (Nx, Ny, Nz), N in [0, mc] per axis, spans
// coarse nodes N and N + 1 (node 0 and mc + 1 on the boundary, value zero)
// and holds the fine nodes 2N + 1 (the midpoint: weight 1/2 on each end) and
// 2N + 2 (coarse node N + 1: weight 1), interior indices 2N and 2N + 1 (the
// latter only for N < mc).  The bilinear/trilinear weights are products of
// these per axis, applied axis by axis; one thread per cell, its two x points
// adjacent in memory.
template <typename T, int D>
__global__ void k_prolong_cells(const cx<T>* __restrict__ ec, int mc, cx<T>* __restrict__ uf, int mf) {
  using C = cx<T>;
  const int Nx = blockIdx.x * BX + threadIdx.x, Ny = blockIdx.y * BY + threadIdx.y;
  const int Nz = (D == 3) ? (int)blockIdx.z : 0;
  if (Nx > mc || Ny > mc) return;
  const T h = (T)0.5;
  // coarse values at the cell's corners: node K -> e[K - 1] inside [1, mc]
  auto ev = [&](int kx, int ky, int kz) -> C {
    const int X = Nx + kx, Y = Ny + ky, Z = Nz + kz;
    if (X < 1 || X > mc || Y < 1 || Y > mc || (D == 3 && (Z < 1 || Z > mc))) return mk<C>(0, 0);
    return ec[((long long)(D == 3 ? Z - 1 : 0) * mc + (Y - 1)) * mc + (X - 1)];
  };
  // along x for each (y, z) corner: mid and coincident values
  C xm[2][2], xc[2][2];
#pragma unroll
  for (int kz = 0; kz < (D == 3 ? 2 : 1); ++kz)
#pragma unroll
    for (int ky = 0; ky < 2; ++ky) {
      const C a = ev(0, ky, kz), b = ev(1, ky, kz);
      xm[kz][ky] = cscale(cadd(a, b), h);
      xc[kz][ky] = b;
    }
  const bool x1 = Nx < mc, y1 = Ny < mc, z1 = (D == 3) ? Nz < mc : false;
  const long long f0 = ((long long)(D == 3 ? 2 * Nz : 0) * mf + 2 * Ny) * mf + 2 * Nx;
  // the cell's fine values first, all in flight together (a load after a
  // store through the same pointer would wait for it)
  C u0[2][2], u1[2][2];
#pragma unroll
  for (int sz = 0; sz < (D == 3 ? 2 : 1); ++sz)
#pragma unroll
    for (int sy = 0; sy < 2; ++sy) {
      const bool in = (sz == 0 || z1) && (sy == 0 || y1);
      const long long f = f0 + ((long long)sz * mf + sy) * mf;
      u0[sz][sy] = in ? uf[f] : mk<C>(0, 0);
      u1[sz][sy] = (in && x1) ? uf[f + 1] : mk<C>(0, 0);
    }
#pragma unroll
  for (int sz = 0; sz < (D == 3 ? 2 : 1); ++sz) {        // fine z: 0 mid, 1 coincident
    if (sz == 1 && !z1) continue;
#pragma unroll
    for (int sy = 0; sy < 2; ++sy) {                      // fine y: 0 mid, 1 coincident
      if (sy == 1 && !y1) continue;
      // along z, then y
      C vm, vc;
      if (D == 3) {
        C ym_m = sz ? xm[1][0] : cscale(cadd(xm[0][0], xm[1][0]), h);
        C ym_c = sz ? xc[1][0] : cscale(cadd(xc[0][0], xc[1][0]), h);
        C yc_m = sz ? xm[1][1] : cscale(cadd(xm[0][1], xm[1][1]), h);
        C yc_c = sz ? xc[1][1] : cscale(cadd(xc[0][1], xc[1][1]), h);
        vm = sy ? yc_m : cscale(cadd(ym_m, yc_m), h);
        vc = sy ? yc_c : cscale(cadd(ym_c, yc_c), h);
      } else {
        vm = sy ? xm[0][1] : cscale(cadd(xm[0][0], xm[0][1]), h);
        vc = sy ? xc[0][1] : cscale(cadd(xc[0][0], xc[0][1]), h);
      }
      const long long f = f0 + ((long long)sz * mf + sy) * mf;
      uf[f] = cadd(u0[sz][sy], vm);
      if (x1) uf[f + 1] = cadd(u1[sz][sy], vc);
    }
  }
}

template <typename T, int D>
__global__ void k_prolong_add(const cx<T>* __restrict__ ec, int mc, cx<T>* __restrict__ uf, int mf) {
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(mf, ix, iy, iz, idx)) return;
  using C = cx<T>;
  int cxi[2], cyi[2], czi[2] = {0, 0};
  T wx[2], wy[2], wz[2] = {(T)1, (T)0};
  int nx = interp_1d<T>(ix, mc, cxi, wx);
  int ny = interp_1d<T>(iy, mc, cyi, wy);
  int nz = (D == 3) ? interp_1d<T>(iz, mc, czi, wz) : 1;
  C acc = mk<C>(0, 0);
  for (int a = 0; a < nz; ++a)
    for (int bq = 0; bq < ny; ++bq) {
      long long base = ((long long)czi[a] * mc + cyi[bq]) * mc;
      for (int cq = 0; cq < nx; ++cq) acc = cadd(acc, cscale(ec[base + cxi[cq]], wx[cq] * wy[bq] * wz[a]));
    }
  uf[idx] = cadd(uf[idx], acc);
}

// Coarsest level: u = A_c^{-1} b with the FP64 dense inverse; one CTA, one
// warp per row (lanes split the columns, shuffle reduction).
template <typename T>
__global__ void k_coarse_solve(const cx<T>* __restrict__ inv, int N, const cx<T>* __restrict__ b,
                               cx<T>* __restrict__ u) {
  extern __shared__ unsigned char sb_raw[];
  cx<T>* sb = reinterpret_cast<cx<T>*>(sb_raw);
  for (int j = threadIdx.x; j < N; j += blockDim.x) sb[j] = b[j];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < N; i += nw) {
    cx<T> acc = mk<cx<T>>((T)0, (T)0);
    const cx<T>* row = inv + (long long)i * N;
    for (int j = lane; j < N; j += 32) acc = cadd(acc, cmul(row[j], sb[j]));
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) u[i] = acc;
  }
}

// The FP64 inverse applied in FP64 to an FP32 right-hand side; the product is
// rounded once to FP32 (the mixed solve with its coarsest solve in FP64).
__global__ void k_coarse_solve_f64(const double2* __restrict__ inv, int N, const float2* __restrict__ b,
                                   float2* __restrict__ u) {
  extern __shared__ unsigned char sb_raw[];
  double2* sb = reinterpret_cast<double2*>(sb_raw);
  for (int j = threadIdx.x; j < N; j += blockDim.x) sb[j] = make_double2(b[j].x, b[j].y);
  __syncthreads();
  // four consecutive lanes per row (columns j = p mod 4), fused multiply-add
  // chains, two shuffles: FP64 work is scarce on this part
  for (int t = threadIdx.x; t < ((4 * N + 31) & ~31); t += blockDim.x) {
    const int i = t >> 2, part = t & 3;
    double re = 0.0, im = 0.0;
    if (i < N) {
      const double2* row = inv + (long long)i * N;
      for (int j = part; j < N; j += 4) {
        const double2 a = row[j], x = sb[j];
        re = fma(a.x, x.x, fma(-a.y, x.y, re));
        im = fma(a.x, x.y, fma(a.y, x.x, im));
      }
    }
    re += __shfl_xor_sync(0xffffffffu, re, 1);
    im += __shfl_xor_sync(0xffffffffu, im, 1);
    re += __shfl_xor_sync(0xffffffffu, re, 2);
    im += __shfl_xor_sync(0xffffffffu, im, 2);
    if (i < N && part == 0) u[i] = make_float2(__double2float_rn(re), __double2float_rn(im));
  }
}

// ---- reductions ------------------------------------------------------------
// Block-wide reduction; the result is valid in thread 0.
template <typename V, typename Op>
__device__ __forceinline__ V block_reduce(V v, Op op, V* sh, V identity) {
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  if (w == 0) {
    v = (l < nw) ? sh[l] : identity;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

struct AddOp { __device__ double operator()(double a, double b) const { return a + b; } };
struct MaxIOp { __device__ int operator()(int a, int b) const { return a > b ? a : b; } };

constexpr int RED_THREADS = 256;

template <typename T>
__global__ void k_norm_partial(const cx<T>* __restrict__ v, long long N, double scale,
                               double* __restrict__ partial) {
  pdl_prologue();
  __shared__ double sh[32];
  double acc = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double a = (double)v[i].x * scale, b = (double)v[i].y * scale;
    acc = fma(a, a, fma(b, b, acc));
  }
  acc = block_reduce(acc, AddOp(), sh, 0.0);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_norm_finish(const double* __restrict__ partial, int nblk, double inv_scale,
                              double* __restrict__ out) {
  pdl_prologue();
  __shared__ double sh[32];
  double acc = 0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += partial[i];
  acc = block_reduce(acc, AddOp(), sh, 0.0);
  if (threadIdx.x == 0) *out = sqrt(acc) * inv_scale;
}

__global__ void k_max_exp(const double2* __restrict__ v, long long N, int* __restrict__ out) {
  __shared__ int sh[32];
  int mx = -2000;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    // frexp's exponent of max(|re|, |im|) from the IEEE fields: -2000 for zero,
    // 4000 when a component is not finite
    const double2 x = v[i];
    const int Ex = bits::exp_field(x.x), Ey = bits::exp_field(x.y);
    int e;
    if (Ex == 0x7ff || Ey == 0x7ff) e = 4000;
    else {
      const bool nzx = ((unsigned long long)__double_as_longlong(x.x) & bits::ABS_MASK) != 0;
      const bool nzy = ((unsigned long long)__double_as_longlong(x.y) & bits::ABS_MASK) != 0;
      e = max(nzx ? bits::frexp_exp(x.x) : -2000, nzy ? bits::frexp_exp(x.y) : -2000);
    }
    mx = e > mx ? e : mx;
  }
  mx = block_reduce(mx, MaxIOp(), sh, -2000);
  if (threadIdx.x == 0) atomicMax(out, mx);
}

__global__ void k_set_int(int* p, int v) { *p = v; }

// ---- coefficients and right-hand side ----------------------------------------
template <int D>
__device__ __forceinline__ double2 chi_point(const double2* const* tabs, int n_gauss, int m, int ix,
                                             int iy, int iz) {
  double2 chi = make_double2(0, 0);
  for (int g = 0; g < n_gauss; ++g) {
    const double2* t = tabs[g];
    double2 v = cmul(t[ix], t[m + iy]);
    if (D == 3) v = cmul(v, t[2 * m + iz]);
    chi = cadd(chi, v);
  }
  return chi;
}

struct TabPtrs { const double2* p[8]; };

template <int D>
__global__ void k_coefs(TabPtrs tabs, int n_gauss, int m, double k2, double2 c, double2* q64,
                        double2* dinv64, float2* q32, float2* dinv32) {
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(m, ix, iy, iz, idx)) return;
  double2 chi = chi_point<D>(tabs.p, n_gauss, m, ix, iy, iz);
  double2 q = make_double2(k2 * (1.0 + chi.x), k2 * chi.y);
  double2 dg = make_double2(2 * D * c.x - q.x, 2 * D * c.y - q.y);
  double den = dg.x * dg.x + dg.y * dg.y;
  double2 di = make_double2(dg.x / den, -dg.y / den);
  q64[idx] = q;
  dinv64[idx] = di;
  q32[idx] = make_float2((float)q.x, (float)q.y);
  dinv32[idx] = make_float2((float)di.x, (float)di.y);
}

// coarse q at the coarse nodes, which are fine nodes 2 I + 1 per axis
template <int D>
__global__ void k_inject_q(const double2* __restrict__ qf, int mf, double2* __restrict__ qc, int mc) {
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(mc, ix, iy, iz, idx)) return;
  const long long f = ((long long)(D == 3 ? 2 * iz + 1 : 0) * mf + 2 * iy + 1) * mf + 2 * ix + 1;
  qc[idx] = qf[f];
}

// 1/d = 1/(2d c - q) and the FP32 copies from a level's q64
template <int D>
__global__ void k_coefs_from_q(const double2* __restrict__ q64, int m, double2 c, double2* dinv64, float2* q32,
                               float2* dinv32) {
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(m, ix, iy, iz, idx)) return;
  const double2 q = q64[idx];
  const double2 dg = make_double2(2 * D * c.x - q.x, 2 * D * c.y - q.y);
  const double den = dg.x * dg.x + dg.y * dg.y;
  const double2 di = make_double2(dg.x / den, -dg.y / den);
  dinv64[idx] = di;
  q32[idx] = make_float2((float)q.x, (float)q.y);
  dinv32[idx] = make_float2((float)di.x, (float)di.y);
}

template <int D>
__global__ void k_rhs(TabPtrs tabs, int n_gauss, const double2* __restrict__ uinc, int m, double k2,
                      double2* __restrict__ b) {
  // chi u_in = sum_g prod_c (E_{g,c} U_c): each axis' Gaussian factor is paired
  // with its incident-wave factor first, so no partial product leaves the
  // FP64 range when chi u_in itself does not.  The pairs for the block's 32
  // columns, 8 rows (and plane) are formed once per block, and so are the
  // row factors k^2 (E_y U_y)(E_z U_z): a node costs one complex product per
  // Gaussian (this pass runs on the FP64 pipe, 1/61 of the FP32 rate here).
  __shared__ double2 px[8][BX], py[8][BY], pz[8];
  const int t = threadIdx.y * BX + threadIdx.x;
  for (int i = t; i < n_gauss * (BX + BY + 1); i += BX * BY) {
    const int g = i / (BX + BY + 1), r = i % (BX + BY + 1);
    const double2* E = tabs.p[g];
    if (r < BX) {
      const int x = blockIdx.x * BX + r;
      px[g][r] = x < m ? cmul(E[x], uinc[x]) : make_double2(0, 0);
    } else if (r < BX + BY) {
      const int y = blockIdx.y * BY + (r - BX);
      py[g][r - BX] = y < m ? cmul(E[m + y], uinc[m + y]) : make_double2(0, 0);
    } else if (D == 3) {
      pz[g] = cmul(E[2 * m + blockIdx.z], uinc[2 * m + blockIdx.z]);
    }
  }
  __syncthreads();
  for (int i = t; i < n_gauss * BY; i += BX * BY) {
    const int g = i / BY, r = i % BY;
    const double2 v = (D == 3) ? cmul(py[g][r], pz[g]) : py[g][r];
    py[g][r] = cscale(v, k2);
  }
  __syncthreads();
  int ix, iy, iz; long long idx;
  if (!thread_point<D>(m, ix, iy, iz, idx)) return;
  double2 acc = n_gauss > 0 ? cmul(px[0][threadIdx.x], py[0][threadIdx.y]) : make_double2(0, 0);
  for (int g = 1; g < n_gauss; ++g) acc = cadd(acc, cmul(px[g][threadIdx.x], py[g][threadIdx.y]));
  b[idx] = acc;
}

// ---- FP64 refinement of the mixed solve (option refine_fp64) -------------------
// r32 = r64 * 2^-e with e = exponent of ||r64||_2 (so |r32| < 1 elementwise).
// The scaling and the rounding to FP32 (to nearest) work on the bit fields,
// keeping the pass off the FP64 pipe (1/61 of the FP32 rate on this part);
// values below FP32's normal range, 2^-126 ||r|| and less, become zero.
__device__ __forceinline__ float d2f_pow2(double v, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned int hi = (unsigned int)(b >> 32);
  const int E = (int)((hi >> 20) & 0x7FF);
  const int Ef = E - e - 1023 + 127;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  if (E == 0x7FF) return mant ? __uint_as_float(0x7FC00000u) : __uint_as_float(0x7F800000u | (hi & 0x80000000u));
  if (E == 0 || Ef <= 0) return 0.f;
  if (Ef >= 255) return __uint_as_float(0x7F800000u | (hi & 0x80000000u));   // beyond FP32's range
  unsigned int f = ((unsigned int)Ef << 23) + (unsigned int)(mant >> 29);
  const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFull), halfway = 0x10000000u;
  f += (rem > halfway || (rem == halfway && (f & 1u))) ? 1u : 0u;
  return __uint_as_float(f | (hi & 0x80000000u));
}

__global__ void k_to32_scaled(const double2* __restrict__ r, long long N, const double* __restrict__ nrm,
                              float2* __restrict__ r32, int* __restrict__ exp_out) {
  pdl_prologue();
  int e;
  frexp(*nrm, &e);
  if (blockIdx.x == 0 && threadIdx.x == 0) *exp_out = e;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = r[i];
    r32[i] = make_float2(d2f_pow2(v.x, e), d2f_pow2(v.y, e));
  }
}

// FP32 value times 2^s as a double, exactly, from the bit fields (zero,
// subnormal input, or a result outside the normal FP64 range take ldexp)
__device__ __forceinline__ double f2d_pow2(float v, int s) {
  const unsigned int b = __float_as_uint(v);
  const int E = (int)((b >> 23) & 0xFFu), Ed = E + 896 + s;
  if (E == 0 || Ed < 1 || Ed > 2046) return ldexp((double)v, s);
  const long long bits = ((long long)(b >> 31) << 63) | ((long long)Ed << 52) |
                         ((long long)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double(bits);
}

__global__ void k_update64(double2* __restrict__ u, const float2* __restrict__ e, long long N,
                           const int* __restrict__ exp_in) {
  pdl_prologue();
  const int s = *exp_in;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 c = e[i];
    double2 v = u[i];
    v.x += f2d_pow2(c.x, s);
    v.y += f2d_pow2(c.y, s);
    u[i] = v;
  }
}

// One pass of the FP64 refinement step (option refine_fp64): the residual
// r = b - A u in FP64 as a chain of fused multiply-adds,
//   r = b - c (2d u - sum_nbr u) + q u,
// its rounding r32 = 2^-s r to FP32 (the right-hand side of the next FP32
// cycles: an exact FP64 scaling and one conversion), and per-block sums of
// |r32|^2 for the norm (within 2^-24 relative of ||2^-s r||, far inside what
// the stopping test resolves).  s is fixed for a solve (the exponent of
// max |b|), so the FP32 values stay below 1 in magnitude.  The kernel is
// bound by instruction issue as much as by the FP64 pipe, so each CTA walks
// grid rows (no index division per point) and nothing else is done per point.
template <int D>
__global__ void k_refine_residual(const double2* __restrict__ u, const double2* __restrict__ b,
                                  const double2* __restrict__ q, double2 c, int m, double scale,
                                  float2* __restrict__ r32, double* __restrict__ partial) {
  pdl_prologue();
  __shared__ double sh[32];
  float acc = 0.f;
  const int nrows = (D == 3) ? m * m : m;
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const double2 z = make_double2(0.0, 0.0);
  if (ix < m) {
    for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
      const int iz = (D == 3) ? row / m : 0;
      const int iy = (D == 3) ? row - iz * m : row;
      const long long i = (long long)row * m + ix;
      const double2 uj = u[i];
      const double2 xl = ix > 0 ? u[i - 1] : z, xr = ix < m - 1 ? u[i + 1] : z;
      const double2 yl = iy > 0 ? u[i - m] : z, yr = iy < m - 1 ? u[i + m] : z;
      double sx = (xl.x + xr.x) + (yl.x + yr.x), sy = (xl.y + xr.y) + (yl.y + yr.y);
      if (D == 3) {
        const long long mm = (long long)m * m;
        const double2 zl = iz > 0 ? u[i - mm] : z, zr = iz < m - 1 ? u[i + mm] : z;
        sx += zl.x + zr.x;
        sy += zl.y + zr.y;
      }
      const double tx = fma((double)(2 * D), uj.x, -sx), ty = fma((double)(2 * D), uj.y, -sy);
      const double2 bj = b[i], qj = q[i];
      const double rx = fma(-c.x, tx, fma(c.y, ty, fma(qj.x, uj.x, fma(-qj.y, uj.y, bj.x))));
      const double ry = fma(-c.x, ty, fma(-c.y, tx, fma(qj.x, uj.y, fma(qj.y, uj.x, bj.y))));
      const float fx = __double2float_rn(rx * scale), fy = __double2float_rn(ry * scale);
      r32[i] = make_float2(fx, fy);
      acc = __fmaf_rn(fx, fx, __fmaf_rn(fy, fy, acc));
    }
  }
  const double tot = block_reduce((double)acc, AddOp(), sh, 0.0);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// u += 2^s e (FP32 correction widened exactly; one FP64 multiply and add per
// component, p2 = 2^s)
__global__ void k_update64_fixed(double2* __restrict__ u, const float2* __restrict__ e, int N, double p2) {
  pdl_prologue();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const float2 c = e[i];
    double2 v = u[i];
    v.x = fma((double)c.x, p2, v.x);
    v.y = fma((double)c.y, p2, v.y);
    u[i] = v;
  }
}

// r32 = 2^-s v rounded to FP32 (the first right-hand side of a solve from zero)
__global__ void k_scale_to32(const double2* __restrict__ v, int N, int s, float2* __restrict__ r32) {
  pdl_prologue();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double2 x = v[i];
    r32[i] = make_float2(d2f_pow2(x.x, s), d2f_pow2(x.y, s));
  }
}

template <typename T>
__global__ void k_zero(cx<T>* v, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = mk<cx<T>>(0, 0);
}

inline dim3 grid_of(int dim, int m) {
  return dim3((m + BX - 1) / BX, (m + BY - 1) / BY, dim == 3 ? m : 1);
}
inline int flat_blocks(long long N) {
  long long b = (N + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define CSFF_DIM_DISPATCH(dim, KERNEL, ...)                                   \
  do {                                                                        \
    if ((dim) == 2) KERNEL<T, 2><<<g, blk, 0, s>>>(__VA_ARGS__);              \
    else KERNEL<T, 3><<<g, blk, 0, s>>>(__VA_ARGS__);                         \
  } while (0)

template <typename T> static const cx<T>* qtab(const Level& L);
template <> const double2* qtab<double>(const Level& L) { return L.q64; }
template <> const float2* qtab<float>(const Level& L) { return L.q32; }
template <typename T> static const cx<T>* dtab(const Level& L);
template <> const double2* dtab<double>(const Level& L) { return L.dinv64; }
template <> const float2* dtab<float>(const Level& L) { return L.dinv32; }

template <typename T>
cudaError_t launch_residual(int dim, const Level& L, const cx<T>* u, const cx<T>* b, cx<T>* r,
                            cudaStream_t s) {
  dim3 g = grid_of(dim, L.m), blk(BX, BY);
  cx<T> c = mk<cx<T>>((T)L.c.x, (T)L.c.y);
  ProfScope ps(mg_family<T>(), s, 3.0 * sizeof(cx<T>) * L.N, 0);
  cudaError_t e = (dim == 2) ? launch_pdl(k_residual<T, 2>, g, blk, 0, s, u, b, qtab<T>(L), c, L.m, r)
                             : launch_pdl(k_residual<T, 3>, g, blk, 0, s, u, b, qtab<T>(L), c, L.m, r);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_jacobi(int dim, const Level& L, double omega, const cx<T>* u, const cx<T>* b,
                          cx<T>* u_out, cudaStream_t s) {
  dim3 g = grid_of(dim, L.m), blk(BX, BY);
  cx<T> c = mk<cx<T>>((T)L.c.x, (T)L.c.y);
  ProfScope ps(mg_family<T>(), s, 3.0 * sizeof(cx<T>) * L.N, 0);
  CSFF_DIM_DISPATCH(dim, k_jacobi, u, b, qtab<T>(L), dtab<T>(L), c, (T)omega, L.m, u_out);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rbgs(int dim, const Level& L, cx<T>* u, const cx<T>* b, cudaStream_t s) {
  dim3 g = grid_of(dim, L.m), blk(BX, BY);
  g.x = ((L.m + 1) / 2 + BX - 1) / BX;          // one thread per point of a colour along x
  cx<T> c = mk<cx<T>>((T)L.c.x, (T)L.c.y);
  ProfScope ps(mg_family<T>(), s, 3.0 * sizeof(cx<T>) * L.N, 0);
  CSFF_DIM_DISPATCH(dim, k_rbgs, u, b, dtab<T>(L), c, L.m, 0);
  CSFF_DIM_DISPATCH(dim, k_rbgs, u, b, dtab<T>(L), c, L.m, 1);
  count_launch(2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(int dim, const Level& F, const Level& C, const cx<T>* r, cx<T>* bc,
                            cudaStream_t s) {
  dim3 g = grid_of(dim, C.m), blk(BX, BY);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * (F.N + C.N), 0);
  CSFF_DIM_DISPATCH(dim, k_restrict, r, F.m, bc, C.m);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(int dim, const Level& F, const Level& C, const cx<T>* ec, cx<T>* u,
                               cudaStream_t s) {
  dim3 g = grid_of(dim, F.m), blk(BX, BY);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * (2.0 * F.N + C.N), 0);
  g = dim3((C.m + 1 + BX - 1) / BX, (C.m + 1 + BY - 1) / BY, dim == 3 ? C.m + 1 : 1);   // coarse cells
  CSFF_DIM_DISPATCH(dim, k_prolong_cells, ec, C.m, u, F.m);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(const cx<T>* inv, int N, const cx<T>* b, cx<T>* u, cudaStream_t s) {
  ProfScope ps(mg_family<T>(), s, sizeof(cx<T>) * (2.0 * N + (double)N * N), 8.0 * N * N);
  k_coarse_solve<T><<<1, 256, (size_t)N * sizeof(cx<T>), s>>>(inv, N, b, u);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve_f64(const double2* inv, int N, const float2* b, float2* u, cudaStream_t s) {
  ProfScope ps(mg_family<float>(), s, sizeof(float2) * 2.0 * N + sizeof(double2) * (double)N * N, 8.0 * N * N);
  k_coarse_solve_f64<<<1, 256, (size_t)N * sizeof(double2), s>>>(inv, N, b, u);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_norm2(const cx<T>* v, long long N, int exp_scale, double* partial, int nblk,
                         double* out, cudaStream_t s) {
  long long need = (N + RED_THREADS - 1) / RED_THREADS;
  int nb = (int)(need < nblk ? (need < 1 ? 1 : need) : nblk);
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * N, 0);
  cudaError_t e = launch_pdl(k_norm_partial<T>, dim3(nb), dim3(RED_THREADS), 0, s, v, N, ldexp(1.0, -exp_scale),
                             partial);
  if (e == cudaSuccess)
    e = launch_pdl(k_norm_finish, dim3(1), dim3(RED_THREADS), 0, s, (const double*)partial, nb,
                   ldexp(1.0, exp_scale), out);
  count_launch(2);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_max_exp(const double2* v, long long N, int* out, cudaStream_t s) {
  k_set_int<<<1, 1, 0, s>>>(out, -2000);
  k_max_exp<<<flat_blocks(N), RED_THREADS, 0, s>>>(v, N, out);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_coefs(int dim, const Level& L, const double2* const* chi_tab, int n_gauss,
                         double k2, cudaStream_t s) {
  TabPtrs t{};
  for (int i = 0; i < n_gauss; ++i) t.p[i] = chi_tab[i];
  dim3 g = grid_of(dim, L.m), blk(BX, BY);
  if (dim == 2)
    k_coefs<2><<<g, blk, 0, s>>>(t, n_gauss, L.m, k2, L.c, L.q64, L.dinv64, L.q32, L.dinv32);
  else
    k_coefs<3><<<g, blk, 0, s>>>(t, n_gauss, L.m, k2, L.c, L.q64, L.dinv64, L.q32, L.dinv32);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_rhs(int dim, int m, const double2* const* chi_tab, int n_gauss,
                       const double2* uinc_tab, double k2, double2* b, cudaStream_t s) {
  TabPtrs t{};
  for (int i = 0; i < n_gauss; ++i) t.p[i] = chi_tab[i];
  dim3 g = grid_of(dim, m), blk(BX, BY);
  if (dim == 2) k_rhs<2><<<g, blk, 0, s>>>(t, n_gauss, uinc_tab, m, k2, b);
  else k_rhs<3><<<g, blk, 0, s>>>(t, n_gauss, uinc_tab, m, k2, b);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_to32_scaled(const double2* r, long long N, const double* norm_dev, float2* r32,
                               int* exp_out, cudaStream_t s) {
  ProfScope ps(PF_MG64, s, 24.0 * N, 0);
  cudaError_t e = launch_pdl(k_to32_scaled, dim3(flat_blocks(N)), dim3(256), 0, s, r, N, norm_dev, r32, exp_out);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_refine_residual(int dim, const Level& L, const double2* u, const double2* b, int s_exp,
                                   float2* r32, double* partial, int nblk, double* out, cudaStream_t s) {
  if (L.N >= (1ll << 31)) return cudaErrorInvalidValue;
  const int gx = (L.m + RED_THREADS - 1) / RED_THREADS;
  const int nrows = dim == 3 ? L.m * L.m : L.m;
  int gy = nblk / gx;
  gy = gy < 1 ? 1 : (gy > nrows ? nrows : gy);
  if (gx * gy > nblk) return cudaErrorInvalidValue;
  ProfScope ps(PF_MG64, s, (16.0 * 3 + 8.0) * L.N, 0);
  const double scale = ldexp(1.0, -s_exp);
  cudaError_t e = (dim == 2)
      ? launch_pdl(k_refine_residual<2>, dim3(gx, gy), dim3(RED_THREADS), 0, s, u, b, (const double2*)L.q64, L.c,
                   L.m, scale, r32, partial)
      : launch_pdl(k_refine_residual<3>, dim3(gx, gy), dim3(RED_THREADS), 0, s, u, b, (const double2*)L.q64, L.c,
                   L.m, scale, r32, partial);
  if (e == cudaSuccess)
    e = launch_pdl(k_norm_finish, dim3(1), dim3(RED_THREADS), 0, s, (const double*)partial, gx * gy,
                   ldexp(1.0, s_exp), out);
  count_launch(2);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_update64_fixed(double2* u, const float2* e, long long N, int s_exp, cudaStream_t s) {
  if (N >= (1ll << 31)) return cudaErrorInvalidValue;
  ProfScope ps(PF_MG64, s, 40.0 * N, 0);
  cudaError_t err = launch_pdl(k_update64_fixed, dim3(flat_blocks(N)), dim3(256), 0, s, u, e, (int)N,
                               ldexp(1.0, s_exp));
  count_launch();
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t launch_scale_to32(const double2* v, long long N, int s_exp, float2* r32, cudaStream_t s) {
  if (N >= (1ll << 31)) return cudaErrorInvalidValue;
  ProfScope ps(PF_MG64, s, 24.0 * N, 0);
  cudaError_t err = launch_pdl(k_scale_to32, dim3(flat_blocks(N)), dim3(256), 0, s, v, (int)N, s_exp, r32);
  count_launch();
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t launch_update64(double2* u, const float2* e, long long N, const int* exp_in,
                            cudaStream_t s) {
  ProfScope ps(PF_MG64, s, 40.0 * N, 0);
  cudaError_t err = launch_pdl(k_update64, dim3(flat_blocks(N)), dim3(256), 0, s, u, e, N, exp_in);
  count_launch();
  return err != cudaSuccess ? err : cudaGetLastError();
}

cudaError_t launch_inject_q(int dim, const Level& F, const Level& C, cudaStream_t s) {
  dim3 g = grid_of(dim, C.m), blk(BX, BY);
  if (dim == 2) k_inject_q<2><<<g, blk, 0, s>>>(F.q64, F.m, C.q64, C.m);
  else k_inject_q<3><<<g, blk, 0, s>>>(F.q64, F.m, C.q64, C.m);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_coefs_from_q(int dim, const Level& L, cudaStream_t s) {
  dim3 g = grid_of(dim, L.m), blk(BX, BY);
  if (dim == 2) k_coefs_from_q<2><<<g, blk, 0, s>>>(L.q64, L.m, L.c, L.dinv64, L.q32, L.dinv32);
  else k_coefs_from_q<3><<<g, blk, 0, s>>>(L.q64, L.m, L.c, L.dinv64, L.q32, L.dinv32);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zero(cx<T>* v, long long N, cudaStream_t s) {
  ProfScope ps(mg_family<T>(), s, (double)sizeof(cx<T>) * N, 0);
  k_zero<T><<<flat_blocks(N), 256, 0, s>>>(v, N);
  count_launch();
  return cudaGetLastError();
}

#define CSFF_INST(T)                                                                                   \
  template cudaError_t launch_residual<T>(int, const Level&, const cx<T>*, const cx<T>*, cx<T>*,       \
                                          cudaStream_t);                                               \
  template cudaError_t launch_jacobi<T>(int, const Level&, double, const cx<T>*, const cx<T>*, cx<T>*, \
                                        cudaStream_t);                                                 \
  template cudaError_t launch_rbgs<T>(int, const Level&, cx<T>*, const cx<T>*, cudaStream_t);         \
  template cudaError_t launch_restrict<T>(int, const Level&, const Level&, const cx<T>*, cx<T>*,       \
                                          cudaStream_t);                                               \
  template cudaError_t launch_prolong_add<T>(int, const Level&, const Level&, const cx<T>*, cx<T>*,    \
                                             cudaStream_t);                                            \
  template cudaError_t launch_coarse_solve<T>(const cx<T>*, int, const cx<T>*, cx<T>*, cudaStream_t);     \
  template cudaError_t launch_norm2<T>(const cx<T>*, long long, int, double*, int, double*,            \
                                       cudaStream_t);                                                  \
  template cudaError_t launch_zero<T>(cx<T>*, long long, cudaStream_t);

CSFF_INST(double)
CSFF_INST(float)

}  // namespace csff
